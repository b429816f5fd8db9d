// Per-slice normal equations of one middle level, by groups of entries that
// share an environment (CUDA cores, rank R = 4 or 8).
//
// Inside a slice k of S^{m+1}, the left environment h_m of an entry depends
// only on its row i (the column bits it passed, j_0 .. j_{m-2}, are fixed by
// the slice) and the right environment w_m only on its column j.  With the
// design a_e = h_e (x) w_e (a[a R + c] = h_a w_c),
//   K[(a,c),(a',c')] = sum_e conj(h_a w_c) h_a' w_c'
//                    = sum_g X_g[a][a'] Y_g[c][c'],
//   y[(a,c)]         = sum_g xv_g[a] yv_g[c],
// where a group g is the entries of one row (X = conj(h) h^T, xv = conj(h),
// Y = sum_e conj(w_e) w_e^T, yv = sum_e conj(w_e) t_e) or of one column
// (Y = conj(w) w^T, yv = conj(w), X = sum_e conj(h_e) h_e^T,
// xv = sum_e conj(h_e) t_e).  The slice's sums (Alg. 1, middle factors) are
// the same; the rank-one update per entry becomes one per group, which at
// the outer levels (few rows or few columns per slice) is many times fewer.
//
// Layout: the level order keeps each group contiguous; gseg[k] is the first
// group of slice k, gstart[g] the first position of group g.  Work per slice
// as in k_mid_gram: 4 x 4 complex tiles of the lower triangle of K owned by
// threads (tile I, J: rows a = 4I / R, c = 4I mod R + u; columns likewise),
// chunks of 32 groups formed into a double-buffered ring by all threads,
// chunk partials Kahan-folded in the precision form.  Same output record.
#pragma once

#include "bfc_kernels.cuh"

namespace bfc {

template <typename V> __device__ __forceinline__ V make_conj(V a)
{
    a.y = -a.y;
    return a;
}

template <typename T, int R> struct GrpCfg {
    static_assert(R == 4 || R == 8, "grouped Gram tiles need R in {4, 8}");
    static constexpr int D = R * R;
    static constexpr int NB = D / 4;
    static constexpr int NT = NB * (NB + 1) / 2;
    static constexpr int CG = 16;                          // groups per chunk
    static constexpr int GT = (160 / NT) < 1 ? 1 : (160 / NT);
    static constexpr int G = GT > CG ? CG : GT;            // thread groups over the chunk's groups
    static constexpr int NTH = ((NT * G + 31) / 32) * 32;
    static constexpr int FOLD = 2;
    static constexpr bool COMP = sizeof(T) == 4;
    static constexpr int NPK = D * (D + 1) / 2;
    static constexpr int GS = 2 * D + 2 * R;               // X, Y, xv, yv per group
    static constexpr int CSTRIDE = 40;
    static constexpr size_t VS = sizeof(typename cvec<T>::type);
    static constexpr size_t RING = 2 * (size_t)CG * GS * VS;
    static constexpr size_t CBYTES = COMP ? (size_t)NTH * CSTRIDE * sizeof(float) : 0;
    static constexpr size_t KBYTES = G > 1 ? (size_t)(NPK + D) * sizeof(double2) : 0;
    static constexpr size_t UBYTES = ((CBYTES > KBYTES ? CBYTES : KBYTES) + 15) / 16 * 16;
    static constexpr size_t SMEM = RING + UBYTES + 16;
    static constexpr int MINB0 = 65536 / (NTH * 128);
    static constexpr int MINB = MINB0 < 1 ? 1 : (MINB0 > 3 ? 3 : MINB0);
};

template <typename T, int R>
__global__ void __launch_bounds__(GrpCfg<T, R>::NTH, GrpCfg<T, R>::MINB)
k_mid_gram_grp(const typename cvec<T>::type* __restrict__ H, const typename cvec<T>::type* __restrict__ Wm,
               const typename cvec<T>::type* __restrict__ tv, const int32_t* __restrict__ gseg,
               const int32_t* __restrict__ gstart, int by_col, typename cvec<T>::type* __restrict__ rec, int S)
{
    typedef typename cvec<T>::type V;
    typedef GrpCfg<T, R> C;
    constexpr int D = C::D, NPK = C::NPK, CG = C::CG, NTH = C::NTH, GS = C::GS;
    extern __shared__ __align__(16) unsigned char smem[];
    V* ring = (V*)smem;                           // [2][CG][GS]
    unsigned char* U = smem + C::RING;
    float* c_s = (float*)U;                       // compensation [CSTRIDE][NTH]
    double2* Kacc = (double2*)U;                  // thread-group reduction (G > 1)

    const int tid = threadIdx.x;
    const bool worker = tid < C::NT * C::G;
    const int grp = tid / C::NT, tile = tid - (tid / C::NT) * C::NT;
    int I = 0;
    while ((I + 1) * (I + 2) / 2 <= tile) ++I;
    const int J = tile - I * (I + 1) / 2;
    const bool diag = (I == J);
    const int aI = (4 * I) / R, cI = (4 * I) % R, aJ = (4 * J) / R, cJ = (4 * J) % R;

    // the X, Y, xv, yv of groups [g, g + cnt) into ring buffer rb
    auto form = [&](int rb, int g, int cnt) {
        V* buf = ring + (size_t)rb * CG * GS;
        for (int idx = tid; idx < CG * GS; idx += NTH) {
            const int gi = idx / GS, x = idx - gi * GS;
            V val = czero<V>();
            if (gi < cnt) {
                const int e0 = gstart[g + gi], e1 = gstart[g + gi + 1];
                // shared vector s (h of a row group, w of a column group) and
                // the summed vectors u of the entries (w, resp. h)
                const V* Sv = by_col ? Wm : H;
                const V* Uv = by_col ? H : Wm;
                // X (the h side) occupies [0, D), Y (the w side) [D, 2D),
                // xv [2D, 2D + R), yv [2D + R, 2D + 2R)
                const bool hside = x < D || (x >= 2 * D && x < 2 * D + R);
                const bool shared_side = by_col ? !hside : hside;
                if (x < 2 * D) {
                    const int xx = x < D ? x : x - D, p = xx / R, q = xx - (xx / R) * R;
                    if (shared_side) {
                        val = cmul(make_conj(Sv[(size_t)e0 * R + p]), Sv[(size_t)e0 * R + q]);
                    } else {
                        for (int e = e0; e < e1; ++e) cmacc(val, Uv[(size_t)e * R + p], Uv[(size_t)e * R + q]);
                    }
                } else {
                    const int p = x < 2 * D + R ? x - 2 * D : x - 2 * D - R;
                    if (shared_side) {
                        val = make_conj(Sv[(size_t)e0 * R + p]);
                    } else {
                        for (int e = e0; e < e1; ++e) cmacc(val, Uv[(size_t)e * R + p], tv[e]);
                    }
                }
            }
            buf[idx] = val;
        }
    };

    for (int k = blockIdx.x; k < S; k += gridDim.x) {
        const int g0 = gseg[k], g1 = gseg[k + 1];
        const int nch = (g1 - g0 + CG - 1) / CG;
        V acc[4][4], sum[4][4], yacc[4], ysum[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            yacc[u] = czero<V>();
            ysum[u] = czero<V>();
#pragma unroll
            for (int v = 0; v < 4; ++v) { acc[u][v] = czero<V>(); sum[u][v] = czero<V>(); }
        }
        __syncthreads();  // previous slice done with every shared buffer
        if (C::COMP && worker)
            for (int x = 0; x < C::CSTRIDE; ++x) c_s[x * NTH + tid] = 0.0f;
        if (nch > 0) form(0, g0, min(CG, g1 - g0));
        int pend = 0;
        for (int c = 0; c < nch; ++c) {
            const int gb = g0 + c * CG;
            const int cnt = min(CG, g1 - gb);
            __syncthreads();  // chunk c formed (ring c & 1); ring (c + 1) & 1 free
            if (c + 1 < nch) form((c + 1) & 1, gb + CG, min(CG, g1 - gb - CG));
            if (worker) {
                const V* buf = ring + (size_t)(c & 1) * CG * GS;
                for (int gi = grp; gi < cnt; gi += C::G) {
                    const V* gr = buf + gi * GS;
                    const V x = gr[aI * R + aJ];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        V yr[4];
                        load4(yr, gr + D + (cI + u) * R + cJ);
#pragma unroll
                        for (int v = 0; v < 4; ++v) cmac(acc[u][v], x, yr[v]);
                    }
                    if (diag) {
                        const V xv = gr[2 * D + aI];
#pragma unroll
                        for (int u = 0; u < 4; ++u) cmac(yacc[u], xv, gr[2 * D + R + cI + u]);
                    }
                }
                if (C::COMP && (++pend == C::FOLD || c + 1 == nch)) {
                    pend = 0;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            float sx = (float)sum[u][v].x, sy = (float)sum[u][v].y;
                            float& cx = c_s[(2 * (u * 4 + v)) * NTH + tid];
                            float& cy = c_s[(2 * (u * 4 + v) + 1) * NTH + tid];
                            kahan(sx, cx, (float)acc[u][v].x);
                            kahan(sy, cy, (float)acc[u][v].y);
                            sum[u][v].x = sx; sum[u][v].y = sy;
                            acc[u][v] = czero<V>();
                        }
                        if (diag) {
                            float sx = (float)ysum[u].x, sy = (float)ysum[u].y;
                            float& cx = c_s[(32 + 2 * u) * NTH + tid];
                            float& cy = c_s[(32 + 2 * u + 1) * NTH + tid];
                            kahan(sx, cx, (float)yacc[u].x);
                            kahan(sy, cy, (float)yacc[u].y);
                            ysum[u].x = sx; ysum[u].y = sy;
                            yacc[u] = czero<V>();
                        }
                    }
                }
            }
        }
        if (C::COMP && worker) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    acc[u][v].x = sum[u][v].x - c_s[(2 * (u * 4 + v)) * NTH + tid];
                    acc[u][v].y = sum[u][v].y - c_s[(2 * (u * 4 + v) + 1) * NTH + tid];
                }
                if (diag) {
                    yacc[u].x = ysum[u].x - c_s[(32 + 2 * u) * NTH + tid];
                    yacc[u].y = ysum[u].y - c_s[(32 + 2 * u + 1) * NTH + tid];
                }
            }
        }
        V* out = rec + (size_t)k * (NPK + D);
        if (C::G == 1) {
            if (worker) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int p = I * 4 + u;
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int q = J * 4 + v;
                        if (q <= p) out[tri(p, q)] = acc[u][v];
                    }
                    if (diag) out[NPK + p] = yacc[u];
                }
            }
        } else {
            __syncthreads();  // compensation reads done before Kacc overwrites them
            for (int q = tid; q < NPK + D; q += NTH) Kacc[q] = make_double2(0.0, 0.0);
            __syncthreads();
            for (int g = 0; g < C::G; ++g) {  // deterministic order over the thread groups
                if (worker && grp == g) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int p = I * 4 + u;
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const int q = J * 4 + v;
                            if (q <= p) {
                                Kacc[tri(p, q)].x += (double)acc[u][v].x;
                                Kacc[tri(p, q)].y += (double)acc[u][v].y;
                            }
                        }
                        if (diag) {
                            Kacc[NPK + p].x += (double)yacc[u].x;
                            Kacc[NPK + p].y += (double)yacc[u].y;
                        }
                    }
                }
                __syncthreads();
            }
            for (int q = tid; q < NPK + D; q += NTH) out[q] = from_d2<V>(Kacc[q]);
        }
    }
}

}  // namespace bfc
