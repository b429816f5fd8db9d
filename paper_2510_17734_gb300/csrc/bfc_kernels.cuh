// Device kernels of the butterfly-completion hot path (Alg. 1 / Eqs.
// grad_butterfly_*), templated on the compute type T (float for the
// precision form, double for the FP64 path) and the rank R.
//
// Orders and buffers (see bfc_internal.h): every training entry has a
// position in each level order l = 0..L+1.  Level-l work reads contiguous
// per-position data (environment vectors, values) of its own order and
// scatters what the next level needs through the precomputed maps nxt / prv.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bfc {

template <typename T> struct cvec;
template <> struct cvec<float> { typedef float2 type; };
template <> struct cvec<double> { typedef double2 type; };

template <typename V> __device__ __forceinline__ V czero() { V v; v.x = 0; v.y = 0; return v; }

// a * b
template <typename V> __device__ __forceinline__ V cmul(V a, V b)
{
    V r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// acc += a * b
template <typename V> __device__ __forceinline__ void cmac(V& acc, V a, V b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename V> __device__ __forceinline__ void cmacc(V& acc, V a, V b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

template <typename V> __device__ __forceinline__ double2 to_d2(V a)
{
    return make_double2((double)a.x, (double)a.y);
}
template <typename V> __device__ __forceinline__ V from_d2(double2 a)
{
    V v;
    v.x = (decltype(v.x))a.x;
    v.y = (decltype(v.y))a.y;
    return v;
}

// Kahan step: s + x with running compensation c (true sum ~ s - c).
__device__ __forceinline__ void kahan(float& s, float& c, float x)
{
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Slice id of the middle factor S^{m+1}: psi^{-1}(i_0..i_{L-m}, j_0..j_{m-1}).
__device__ __forceinline__ int slice_of(int pi, int pj, int m, int L)
{
    return ((pi >> (m - 1)) << m) | (pj >> (L - m));
}

// Packed lower-triangular index (p >= q).
__device__ __forceinline__ int tri(int p, int q) { return (p * (p + 1) >> 1) + q; }

// ------------------------------------------------------------------------
// Right environments, one level: w_{m-1} = Z^{m+1}(k) w_m for every entry of
// slice k (Alg. 1: the right vector v, built from the right end).  One CTA
// per slice; the slice is staged in shared memory and read by broadcast.
template <typename T, int R>
__global__ void __launch_bounds__(128)
k_env_right(const typename cvec<T>::type* __restrict__ Win,
            typename cvec<T>::type* __restrict__ Wout,
            const typename cvec<T>::type* __restrict__ Zm,
            const int32_t* __restrict__ seg, const int32_t* __restrict__ prv, int S)
{
    typedef typename cvec<T>::type V;
    __shared__ V z[R * R];
    for (int k = blockIdx.x; k < S; k += gridDim.x) {
        const int s0 = seg[k], s1 = seg[k + 1];
        if (s0 == s1) continue;
        __syncthreads();
        for (int q = threadIdx.x; q < R * R; q += blockDim.x) z[q] = Zm[(size_t)k * R * R + q];
        __syncthreads();
        for (int p = s0 + threadIdx.x; p < s1; p += blockDim.x) {
            V w[R];
#pragma unroll
            for (int c = 0; c < R; ++c) w[c] = Win[(size_t)p * R + c];
            const size_t o = (size_t)prv[p] * R;
#pragma unroll
            for (int a = 0; a < R; ++a) {
                V acc = czero<V>();
#pragma unroll
                for (int c = 0; c < R; ++c) cmac(acc, z[a * R + c], w[c]);
                Wout[o + a] = acc;
            }
        }
    }
}

// w_L = zL(j, :) for the entries in order L.
template <typename T, int R>
__global__ void k_env_init(typename cvec<T>::type* __restrict__ WL,
                           const typename cvec<T>::type* __restrict__ zL,
                           const int32_t* __restrict__ jL, int64_t N)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N * R) return;
    int64_t p = q / R;
    int c = (int)(q - p * R);
    WL[q] = zL[(int64_t)jL[p] * R + c];
}

// ------------------------------------------------------------------------
// Serial Hermitian Cholesky solve of a small system (one thread), packed
// lower storage K (D(D+1)/2 entries).  Returns false when a pivot <= tol.
__device__ inline bool chol_solve_serial(double2* K, const double2* y, double2* s, int D,
                                         double tol)
{
    for (int c = 0; c < D; ++c) {
        double d = K[tri(c, c)].x;
        for (int q = 0; q < c; ++q) {
            double2 l = K[tri(c, q)];
            d -= l.x * l.x + l.y * l.y;
        }
        if (!(d > tol)) return false;
        double piv = sqrt(d), inv = 1.0 / piv;
        K[tri(c, c)] = make_double2(piv, 0.0);
        for (int row = c + 1; row < D; ++row) {
            double2 acc = K[tri(row, c)];
            for (int q = 0; q < c; ++q) {
                double2 a = K[tri(row, q)], bq = K[tri(c, q)];
                // acc -= a * conj(bq)
                acc.x -= a.x * bq.x + a.y * bq.y;
                acc.y -= a.y * bq.x - a.x * bq.y;
            }
            K[tri(row, c)] = make_double2(acc.x * inv, acc.y * inv);
        }
    }
    for (int row = 0; row < D; ++row) {
        double2 acc = y[row];
        for (int q = 0; q < row; ++q) {
            double2 l = K[tri(row, q)], z = s[q];
            acc.x -= l.x * z.x - l.y * z.y;
            acc.y -= l.x * z.y + l.y * z.x;
        }
        double inv = 1.0 / K[tri(row, row)].x;
        s[row] = make_double2(acc.x * inv, acc.y * inv);
    }
    for (int row = D - 1; row >= 0; --row) {
        double2 acc = s[row];
        for (int q = row + 1; q < D; ++q) {
            double2 l = K[tri(q, row)], z = s[q];
            // acc -= conj(l) * z
            acc.x -= l.x * z.x + l.y * z.y;
            acc.y -= l.x * z.y - l.y * z.x;
        }
        double inv = 1.0 / K[tri(row, row)].x;
        s[row] = make_double2(acc.x * inv, acc.y * inv);
    }
    return true;
}

// ------------------------------------------------------------------------
// Outer fibers (S^1 rows when COLS is false, S^{L+2} columns when true):
// one warp per fiber f.  Design vector a_e = A[p] (w_0 for rows, h_{L+1} for
// columns), K = sum conj(a) a^T + lambda I (r x r), y = sum conj(a) t,
// solved in FP64 (Alg. 1, first and last branches, complex form).
// Rows then write h_1 = z1(i, :) for every entry into order 1; columns
// evaluate x = h_{L+1}^T zL(j) and accumulate the training residual.
template <typename T, int R, bool COLS>
__global__ void __launch_bounds__(128)
k_outer(const typename cvec<T>::type* __restrict__ A, const typename cvec<T>::type* __restrict__ tv,
        const int32_t* __restrict__ seg, int nfib, double lambda, double2* __restrict__ zd,
        typename cvec<T>::type* __restrict__ zt, const int32_t* __restrict__ nxt,
        typename cvec<T>::type* __restrict__ Hn, double* __restrict__ err_part,
        unsigned long long* __restrict__ nsing)
{
    typedef typename cvec<T>::type V;
    constexpr bool COMP = sizeof(T) == 4;
    constexpr int NP = R * (R + 1) / 2;
    constexpr int NI = NP + R;
    constexpr int IPL = (NI + 31) / 32;
    constexpr int WPB = 4;  // warps (fibers) per 128-thread block
    __shared__ V a_s[WPB][32 * R];
    __shared__ V t_s[WPB][32];
    __shared__ double2 K_s[WPB][NP];
    __shared__ double2 y_s[WPB][R];
    __shared__ double2 x_s[WPB][R];
    __shared__ int ok_s[WPB];

    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int f = blockIdx.x * WPB + wib;
    if (f >= nfib) return;                       // whole warp leaves; no block barriers below
    const int s0 = seg[f], s1 = seg[f + 1];

    // item -> (p, q) (pair, p >= q) or rhs index
    int ip[IPL], iq[IPL];
#pragma unroll
    for (int u = 0; u < IPL; ++u) {
        int it = lane + 32 * u;
        ip[u] = -1;
        iq[u] = -1;
        if (it < NP) {
            int p = 0;
            while ((p + 1) * (p + 2) / 2 <= it) ++p;
            ip[u] = p;
            iq[u] = it - p * (p + 1) / 2;
        } else if (it < NI) {
            ip[u] = it - NP;
            iq[u] = -2;  // rhs
        }
    }
    V acc[IPL], sum[IPL], cmp[IPL];
#pragma unroll
    for (int u = 0; u < IPL; ++u) { acc[u] = czero<V>(); sum[u] = czero<V>(); cmp[u] = czero<V>(); }

    for (int base = s0; base < s1; base += 32) {
        const int cnt = min(32, s1 - base);
        __syncwarp();
        if (lane < cnt) {
#pragma unroll
            for (int c = 0; c < R; ++c) a_s[wib][lane * R + c] = A[(size_t)(base + lane) * R + c];
            t_s[wib][lane] = tv[base + lane];
        }
        __syncwarp();
        for (int e = 0; e < cnt; ++e) {
            const V* ae = &a_s[wib][e * R];
#pragma unroll
            for (int u = 0; u < IPL; ++u) {
                if (iq[u] >= 0) cmacc(acc[u], ae[ip[u]], ae[iq[u]]);
                else if (iq[u] == -2) cmacc(acc[u], ae[ip[u]], t_s[wib][e]);
            }
        }
        if (COMP) {
#pragma unroll
            for (int u = 0; u < IPL; ++u) {
                float sx = (float)sum[u].x, sy = (float)sum[u].y, cx = (float)cmp[u].x, cy = (float)cmp[u].y;
                kahan(sx, cx, (float)acc[u].x);
                kahan(sy, cy, (float)acc[u].y);
                sum[u].x = sx; sum[u].y = sy; cmp[u].x = cx; cmp[u].y = cy;
                acc[u] = czero<V>();
            }
        }
    }
    // assemble the system in FP64
#pragma unroll
    for (int u = 0; u < IPL; ++u) {
        double2 v = COMP ? make_double2((double)sum[u].x - (double)cmp[u].x,
                                        (double)sum[u].y - (double)cmp[u].y)
                         : to_d2(acc[u]);
        if (iq[u] >= 0) K_s[wib][tri(ip[u], iq[u])] = v;
        else if (iq[u] == -2) y_s[wib][ip[u]] = v;
    }
    __syncwarp();
    if (lane == 0) {
        double trace = 0.0;
        for (int p = 0; p < R; ++p) {
            K_s[wib][tri(p, p)].x += lambda;
            trace += K_s[wib][tri(p, p)].x;
        }
        const double tol = lambda > 0.0 ? 0.0 : 1e-14 * trace;
        ok_s[wib] = chol_solve_serial(K_s[wib], y_s[wib], x_s[wib], R, tol) ? 1 : 0;
        if (!ok_s[wib]) atomicAdd(nsing, 1ull);
    }
    __syncwarp();
    const bool ok = ok_s[wib] != 0;
    if (ok && lane < R) {
        zd[(size_t)f * R + lane] = x_s[wib][lane];
        zt[(size_t)f * R + lane] = from_d2<V>(x_s[wib][lane]);
    }
    __syncwarp();
    V zf[R];
#pragma unroll
    for (int c = 0; c < R; ++c) zf[c] = ok ? from_d2<V>(x_s[wib][c]) : zt[(size_t)f * R + c];

    if (!COLS) {
        for (int p = s0 + lane; p < s1; p += 32) {
            const size_t o = (size_t)nxt[p] * R;
#pragma unroll
            for (int c = 0; c < R; ++c) Hn[o + c] = zf[c];
        }
    } else {
        double num = 0.0, den = 0.0;
        for (int p = s0 + lane; p < s1; p += 32) {
            V x = czero<V>();
#pragma unroll
            for (int c = 0; c < R; ++c) cmac(x, A[(size_t)p * R + c], zf[c]);
            V t = tv[p];
            double dx = (double)t.x - (double)x.x, dy = (double)t.y - (double)x.y;
            num += dx * dx + dy * dy;
            den += (double)t.x * (double)t.x + (double)t.y * (double)t.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            num += __shfl_xor_sync(0xffffffffu, num, o);
            den += __shfl_xor_sync(0xffffffffu, den, o);
        }
        if (lane == 0) {
            err_part[2 * (size_t)f] = num;
            err_part[2 * (size_t)f + 1] = den;
        }
    }
}

// ------------------------------------------------------------------------
// Middle level m: one CTA per slice k of S^{m+1}.
//   Gram/RHS: a_e = h_m(e) (x) w_m(e) (a[p r + c] = h_p w_c), K = sum conj(a) a^T,
//   y = sum conj(a) t over the slice's entries (Alg. 1 middle branch, complex
//   form).  Threads own 4x4 complex tiles of the lower triangle of K, entries
//   are split over G thread groups and staged in shared memory in chunks of
//   CE.  In float the chunk partials are folded into Kahan-compensated sums.
//   Solve: K + lambda I in FP64, Cholesky (CTA-parallel right-looking on
//   packed storage) + triangular solves; the slice is written row-major.
//   Left update: h_{m+1}(e) = h_m(e)^T Z^{m+1}(k) scattered into order m+1.
template <typename T, int R> struct MidCfg {
    static constexpr int D = R * R;
    static constexpr int DP = (D + 3) / 4 * 4;
    static constexpr int NB = DP / 4;
    static constexpr int NT = NB * (NB + 1) / 2;
    static constexpr int CE = (DP <= 36) ? 64 : 32;
    static constexpr int GT = (288 / NT) < 1 ? 1 : (288 / NT);
    static constexpr int G = GT > CE ? CE : GT;
    static constexpr int NTH = ((NT * G + 31) / 32) * 32;
    static constexpr bool COMP = sizeof(T) == 4;
    static constexpr int CSTRIDE = 40;  // floats of compensation per worker thread
    static constexpr size_t KBYTES = (size_t)D * (D + 1) / 2 * sizeof(double2);
    static constexpr size_t CBYTES = COMP ? (size_t)NTH * CSTRIDE * sizeof(float) : 0;
    static constexpr size_t UBYTES = KBYTES > CBYTES ? KBYTES : CBYTES;
    static constexpr size_t VS = sizeof(typename cvec<T>::type);
    static constexpr size_t SMEM = (size_t)CE * DP * VS + (size_t)CE * VS + ((UBYTES + 15) / 16) * 16 +
                                   2 * (size_t)DP * sizeof(double2) + (size_t)DP * VS + 16;
};

template <typename T, int R>
__global__ void __launch_bounds__(MidCfg<T, R>::NTH)
k_mid(const typename cvec<T>::type* __restrict__ H, const typename cvec<T>::type* __restrict__ Wm,
      const typename cvec<T>::type* __restrict__ tv, const int32_t* __restrict__ seg,
      const int32_t* __restrict__ nxt, typename cvec<T>::type* __restrict__ Hn,
      double2* __restrict__ Zd, typename cvec<T>::type* __restrict__ Zt, double lambda,
      unsigned long long* __restrict__ nsing, int S)
{
    typedef typename cvec<T>::type V;
    typedef MidCfg<T, R> C;
    constexpr int D = C::D, DP = C::DP;
    extern __shared__ __align__(16) unsigned char smem[];
    V* a_s = (V*)smem;
    V* t_s = a_s + C::CE * DP;
    unsigned char* U = (unsigned char*)(t_s + C::CE);
    double2* K_s = (double2*)U;
    float* c_s = (float*)U;
    double2* y_s = (double2*)(U + ((C::UBYTES + 15) / 16) * 16);
    double2* x_s = y_s + DP;
    V* zt_s = (V*)(x_s + DP);
    int* flag_s = (int*)(zt_s + DP);

    const int tid = threadIdx.x;
    const int nth = blockDim.x;
    const bool worker = tid < C::NT * C::G;
    const int grp = tid / C::NT, tile = tid - (tid / C::NT) * C::NT;
    int I = 0;
    while ((I + 1) * (I + 2) / 2 <= tile) ++I;
    const int J = tile - I * (I + 1) / 2;
    const bool diag = (I == J);

    for (int k = blockIdx.x; k < S; k += gridDim.x) {
        const int s0 = seg[k], s1 = seg[k + 1];
        V acc[4][4], sum[4][4], yacc[4], ysum[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            yacc[u] = czero<V>();
            ysum[u] = czero<V>();
#pragma unroll
            for (int v = 0; v < 4; ++v) { acc[u][v] = czero<V>(); sum[u][v] = czero<V>(); }
        }
        __syncthreads();  // previous slice done with the shared buffers
        if (C::COMP && worker)
            for (int x = 0; x < C::CSTRIDE; ++x) c_s[x * C::NTH + tid] = 0.0f;

        for (int base = s0; base < s1; base += C::CE) {
            const int cnt = min(C::CE, s1 - base);
            __syncthreads();
            for (int idx = tid; idx < cnt * DP; idx += nth) {
                const int e = idx / DP, q = idx - e * DP;
                V a = czero<V>();
                if (q < D) {
                    const int pa = q / R, pc = q - pa * R;
                    a = cmul(H[(size_t)(base + e) * R + pa], Wm[(size_t)(base + e) * R + pc]);
                }
                a_s[e * DP + q] = a;
            }
            for (int e = tid; e < cnt; e += nth) t_s[e] = tv[base + e];
            __syncthreads();
            if (worker) {
                for (int e = grp; e < cnt; e += C::G) {
                    const V* ae = a_s + e * DP;
                    V ap[4], aq[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) { ap[u] = ae[I * 4 + u]; aq[u] = ae[J * 4 + u]; }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) cmacc(acc[u][v], ap[u], aq[v]);
                    if (diag) {
                        const V te = t_s[e];
#pragma unroll
                        for (int u = 0; u < 4; ++u) cmacc(yacc[u], ap[u], te);
                    }
                }
                if (C::COMP) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            float sx = (float)sum[u][v].x, sy = (float)sum[u][v].y;
                            float cx = c_s[(2 * (u * 4 + v)) * C::NTH + tid];
                            float cy = c_s[(2 * (u * 4 + v) + 1) * C::NTH + tid];
                            kahan(sx, cx, (float)acc[u][v].x);
                            kahan(sy, cy, (float)acc[u][v].y);
                            sum[u][v].x = sx; sum[u][v].y = sy;
                            c_s[(2 * (u * 4 + v)) * C::NTH + tid] = cx;
                            c_s[(2 * (u * 4 + v) + 1) * C::NTH + tid] = cy;
                            acc[u][v] = czero<V>();
                        }
                        if (diag) {
                            float sx = (float)ysum[u].x, sy = (float)ysum[u].y;
                            float cx = c_s[(32 + 2 * u) * C::NTH + tid];
                            float cy = c_s[(32 + 2 * u + 1) * C::NTH + tid];
                            kahan(sx, cx, (float)yacc[u].x);
                            kahan(sy, cy, (float)yacc[u].y);
                            ysum[u].x = sx; ysum[u].y = sy;
                            c_s[(32 + 2 * u) * C::NTH + tid] = cx;
                            c_s[(32 + 2 * u + 1) * C::NTH + tid] = cy;
                            yacc[u] = czero<V>();
                        }
                    }
                }
            }
        }
        __syncthreads();
        // final per-thread values (compensated in float), held in acc / yacc
        if (worker) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    if (C::COMP) {
                        acc[u][v].x = sum[u][v].x - c_s[(2 * (u * 4 + v)) * C::NTH + tid];
                        acc[u][v].y = sum[u][v].y - c_s[(2 * (u * 4 + v) + 1) * C::NTH + tid];
                    }
                }
                if (C::COMP && diag) {
                    yacc[u].x = ysum[u].x - c_s[(32 + 2 * u) * C::NTH + tid];
                    yacc[u].y = ysum[u].y - c_s[(32 + 2 * u + 1) * C::NTH + tid];
                }
            }
        }
        __syncthreads();
        for (int q = tid; q < D * (D + 1) / 2; q += nth) K_s[q] = make_double2(0.0, 0.0);
        for (int q = tid; q < DP; q += nth) y_s[q] = make_double2(0.0, 0.0);
        __syncthreads();
        // deterministic reduction over the entry groups
        for (int g = 0; g < C::G; ++g) {
            if (worker && grp == g) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int p = I * 4 + u;
                    if (p < D) {
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const int q = J * 4 + v;
                            if (q <= p) {
                                double2 cur = K_s[tri(p, q)];
                                cur.x += (double)acc[u][v].x;
                                cur.y += (double)acc[u][v].y;
                                K_s[tri(p, q)] = cur;
                            }
                        }
                        if (diag) {
                            y_s[p].x += (double)yacc[u].x;
                            y_s[p].y += (double)yacc[u].y;
                        }
                    }
                }
            }
            __syncthreads();
        }
        // regularize, pivot threshold
        if (tid == 0) {
            double trace = 0.0;
            for (int p = 0; p < D; ++p) {
                K_s[tri(p, p)].x += lambda;
                trace += K_s[tri(p, p)].x;
            }
            flag_s[0] = 1;
            reinterpret_cast<double*>(flag_s + 2)[0] = lambda > 0.0 ? 0.0 : 1e-14 * trace;
        }
        __syncthreads();
        const double tol = reinterpret_cast<double*>(flag_s + 2)[0];
        // right-looking Cholesky K = L L^H on packed lower storage
        for (int c = 0; c < D; ++c) {
            if (tid == 0) {
                const double d = K_s[tri(c, c)].x;
                if (d > tol) {
                    K_s[tri(c, c)] = make_double2(sqrt(d), 0.0);
                } else {
                    flag_s[0] = 0;
                }
            }
            __syncthreads();
            if (!flag_s[0]) break;
            const double inv = 1.0 / K_s[tri(c, c)].x;
            for (int row = c + 1 + tid; row < D; row += nth) {
                double2 l = K_s[tri(row, c)];
                K_s[tri(row, c)] = make_double2(l.x * inv, l.y * inv);
            }
            __syncthreads();
            const int m = D - c - 1;
            const int npairs = m * (m + 1) / 2;
            for (int idx = tid; idx < npairs; idx += nth) {
                int rr = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
                while ((rr + 1) * (rr + 2) / 2 <= idx) ++rr;
                while (rr * (rr + 1) / 2 > idx) --rr;
                const int qq = idx - rr * (rr + 1) / 2;
                const int r_ = c + 1 + rr, q_ = c + 1 + qq;
                const double2 a = K_s[tri(r_, c)], bq = K_s[tri(q_, c)];
                double2 cur = K_s[tri(r_, q_)];
                // cur -= a * conj(bq)
                cur.x -= a.x * bq.x + a.y * bq.y;
                cur.y -= a.y * bq.x - a.x * bq.y;
                K_s[tri(r_, q_)] = cur;
            }
            __syncthreads();
        }
        const bool ok = flag_s[0] != 0;
        if (ok && tid < 32) {
            // forward L z = y (z kept in x_s), then backward L^H x = z
            for (int row = 0; row < D; ++row) {
                double px = 0.0, py = 0.0;
                for (int q = tid; q < row; q += 32) {
                    const double2 l = K_s[tri(row, q)], z = x_s[q];
                    px += l.x * z.x - l.y * z.y;
                    py += l.x * z.y + l.y * z.x;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    px += __shfl_xor_sync(0xffffffffu, px, o);
                    py += __shfl_xor_sync(0xffffffffu, py, o);
                }
                if (tid == 0) {
                    const double inv = 1.0 / K_s[tri(row, row)].x;
                    x_s[row] = make_double2((y_s[row].x - px) * inv, (y_s[row].y - py) * inv);
                }
                __syncwarp();
            }
            for (int row = D - 1; row >= 0; --row) {
                double px = 0.0, py = 0.0;
                for (int q = row + 1 + tid; q < D; q += 32) {
                    const double2 l = K_s[tri(q, row)], z = x_s[q];
                    px += l.x * z.x + l.y * z.y;
                    py += l.x * z.y - l.y * z.x;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    px += __shfl_xor_sync(0xffffffffu, px, o);
                    py += __shfl_xor_sync(0xffffffffu, py, o);
                }
                if (tid == 0) {
                    const double inv = 1.0 / K_s[tri(row, row)].x;
                    x_s[row] = make_double2((x_s[row].x - px) * inv, (x_s[row].y - py) * inv);
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (!ok && tid == 0) atomicAdd(nsing, 1ull);
        for (int q = tid; q < D; q += nth) {
            if (ok) {
                const double2 s = x_s[q];
                Zd[(size_t)k * D + q] = s;
                const V st = from_d2<V>(s);
                Zt[(size_t)k * D + q] = st;
                zt_s[q] = st;
            } else {
                zt_s[q] = Zt[(size_t)k * D + q];
            }
        }
        __syncthreads();
        // left environment update into the next order
        for (int p = s0 + tid; p < s1; p += nth) {
            V h[R];
#pragma unroll
            for (int a = 0; a < R; ++a) h[a] = H[(size_t)p * R + a];
            const size_t o = (size_t)nxt[p] * R;
#pragma unroll
            for (int c = 0; c < R; ++c) {
                V acc2 = czero<V>();
#pragma unroll
                for (int a = 0; a < R; ++a) cmac(acc2, h[a], zt_s[a * R + c]);
                Hn[o + c] = acc2;
            }
        }
    }
}

// ------------------------------------------------------------------------
// Entry evaluation x = z1(i)^T Z^2(k_2) ... Z^{L+1}(k_{L+1}) zL(j)
// (Eq. (BF_tensor_rep)) for arbitrary pairs; optional residual statistics.
template <typename T, int R>
__device__ __forceinline__ typename cvec<T>::type
eval_one(int i, int j, const typename cvec<T>::type* __restrict__ z1,
         const typename cvec<T>::type* __restrict__ Z, const typename cvec<T>::type* __restrict__ zL,
         int L, int b, int64_t S)
{
    typedef typename cvec<T>::type V;
    V h[R];
#pragma unroll
    for (int a = 0; a < R; ++a) h[a] = z1[(size_t)i * R + a];
    const int pi = i / b, pj = j / b;
    for (int m = 1; m <= L; ++m) {
        const V* Zk = Z + ((size_t)(m - 1) * S + slice_of(pi, pj, m, L)) * R * R;
        V nh[R];
#pragma unroll
        for (int c = 0; c < R; ++c) {
            V acc = czero<V>();
#pragma unroll
            for (int a = 0; a < R; ++a) cmac(acc, h[a], Zk[a * R + c]);
            nh[c] = acc;
        }
#pragma unroll
        for (int c = 0; c < R; ++c) h[c] = nh[c];
    }
    V x = czero<V>();
#pragma unroll
    for (int c = 0; c < R; ++c) cmac(x, h[c], zL[(size_t)j * R + c]);
    return x;
}

template <typename T, int R>
__global__ void __launch_bounds__(256)
k_eval(const int32_t* __restrict__ ii, const int32_t* __restrict__ jj, int64_t M,
       const typename cvec<T>::type* __restrict__ z1, const typename cvec<T>::type* __restrict__ Z,
       const typename cvec<T>::type* __restrict__ zL, int L, int b, int64_t S,
       double2* __restrict__ out, const double2* __restrict__ tref, double* __restrict__ part)
{
    typedef typename cvec<T>::type V;
    double num = 0.0, den = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < M;
         e += (int64_t)gridDim.x * blockDim.x) {
        const V x = eval_one<T, R>(ii[e], jj[e], z1, Z, zL, L, b, S);
        if (out) out[e] = to_d2(x);
        if (tref) {
            const double2 t = tref[e];
            const double dx = t.x - (double)x.x, dy = t.y - (double)x.y;
            num += dx * dx + dy * dy;
            den += t.x * t.x + t.y * t.y;
        }
    }
    if (part) {
        __shared__ double sn[8], sd[8];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            num += __shfl_xor_sync(0xffffffffu, num, o);
            den += __shfl_xor_sync(0xffffffffu, den, o);
        }
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) { sn[w] = num; sd[w] = den; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, c = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += sn[q]; c += sd[q]; }
            part[2 * blockIdx.x] = a;
            part[2 * blockIdx.x + 1] = c;
        }
    }
}

// ------------------------------------------------------------------------
// Gradient (Eqs. (grad_butterfly_1), (grad_butterfly_l), (grad_butterfly_last)
// with z = x - t): the residual r_e is formed at the row level from the full
// right environment (x = z1(i)^T w_0) and carried with h along the orders.

// Rows: r = z1(i)^T w_0 - t, G1(i) = sum r conj(w_0); writes h_1 = z1(i) and r
// into order 1; per-fiber sum of |r|^2 into part[f].
template <typename T, int R>
__global__ void __launch_bounds__(256)
k_grad_rows(const typename cvec<T>::type* __restrict__ W0, const typename cvec<T>::type* __restrict__ tv,
            const int32_t* __restrict__ seg, int nfib, const typename cvec<T>::type* __restrict__ z1t,
            const int32_t* __restrict__ nxt, typename cvec<T>::type* __restrict__ Hn,
            typename cvec<T>::type* __restrict__ Rn, double2* __restrict__ G1, double* __restrict__ part)
{
    typedef typename cvec<T>::type V;
    const int lane = threadIdx.x & 31;
    const int f = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (f >= nfib) return;
    const int s0 = seg[f], s1 = seg[f + 1];
    V z[R];
#pragma unroll
    for (int c = 0; c < R; ++c) z[c] = z1t[(size_t)f * R + c];
    double2 g[R];
#pragma unroll
    for (int c = 0; c < R; ++c) g[c] = make_double2(0.0, 0.0);
    double fit = 0.0;
    for (int p = s0 + lane; p < s1; p += 32) {
        V w[R];
#pragma unroll
        for (int c = 0; c < R; ++c) w[c] = W0[(size_t)p * R + c];
        V x = czero<V>();
#pragma unroll
        for (int c = 0; c < R; ++c) cmac(x, z[c], w[c]);
        const V t = tv[p];
        V rr;
        rr.x = x.x - t.x;
        rr.y = x.y - t.y;
        fit += (double)rr.x * (double)rr.x + (double)rr.y * (double)rr.y;
#pragma unroll
        for (int c = 0; c < R; ++c) {
            // g += r conj(w)
            g[c].x += (double)rr.x * (double)w[c].x + (double)rr.y * (double)w[c].y;
            g[c].y += (double)rr.y * (double)w[c].x - (double)rr.x * (double)w[c].y;
        }
        const size_t o = (size_t)nxt[p];
#pragma unroll
        for (int c = 0; c < R; ++c) Hn[o * R + c] = z[c];
        Rn[o] = rr;
    }
#pragma unroll
    for (int c = 0; c < R; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            g[c].x += __shfl_xor_sync(0xffffffffu, g[c].x, o);
            g[c].y += __shfl_xor_sync(0xffffffffu, g[c].y, o);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fit += __shfl_xor_sync(0xffffffffu, fit, o);
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < R; ++c) G1[(size_t)f * R + c] = g[c];
        part[f] = fit;
    }
}

// Middle level m: G^{m+1}(k) = sum r conj(h_m (x) w_m); h_{m+1} = h_m^T Z(k); r carried.
template <typename T, int R>
__global__ void __launch_bounds__(128)
k_grad_mid(const typename cvec<T>::type* __restrict__ H, const typename cvec<T>::type* __restrict__ Wm,
           const typename cvec<T>::type* __restrict__ Rc, const int32_t* __restrict__ seg,
           const int32_t* __restrict__ nxt, const typename cvec<T>::type* __restrict__ Zt,
           typename cvec<T>::type* __restrict__ Hn, typename cvec<T>::type* __restrict__ Rn,
           double2* __restrict__ Gm, int S)
{
    typedef typename cvec<T>::type V;
    constexpr int D = R * R;
    constexpr int CH = 64;
    __shared__ V z_s[D];
    __shared__ V h_s[CH * R], w_s[CH * R], r_s[CH];
    for (int k = blockIdx.x; k < S; k += gridDim.x) {
        const int s0 = seg[k], s1 = seg[k + 1];
        __syncthreads();
        for (int q = threadIdx.x; q < D; q += blockDim.x) z_s[q] = Zt[(size_t)k * D + q];
        double2 g[(D + 127) / 128];
#pragma unroll
        for (int u = 0; u < (D + 127) / 128; ++u) g[u] = make_double2(0.0, 0.0);
        for (int base = s0; base < s1; base += CH) {
            const int cnt = min(CH, s1 - base);
            __syncthreads();
            for (int q = threadIdx.x; q < cnt * R; q += blockDim.x) {
                h_s[q] = H[(size_t)base * R + q];
                w_s[q] = Wm[(size_t)base * R + q];
            }
            for (int q = threadIdx.x; q < cnt; q += blockDim.x) r_s[q] = Rc[base + q];
            __syncthreads();
            // gradient components owned by threads
#pragma unroll
            for (int u = 0; u < (D + 127) / 128; ++u) {
                const int q = threadIdx.x + 128 * u;
                if (q < D) {
                    const int pa = q / R, pc = q - pa * R;
                    V acc = czero<V>();
                    for (int e = 0; e < cnt; ++e) {
                        const V a = cmul(h_s[e * R + pa], w_s[e * R + pc]);
                        cmacc(acc, a, r_s[e]);   // conj(a) r
                    }
                    g[u].x += (double)acc.x;
                    g[u].y += (double)acc.y;
                }
            }
            // carry h and r into the next order
            for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
                const size_t o = (size_t)nxt[base + e];
#pragma unroll
                for (int c = 0; c < R; ++c) {
                    V acc2 = czero<V>();
#pragma unroll
                    for (int a = 0; a < R; ++a) cmac(acc2, h_s[e * R + a], z_s[a * R + c]);
                    Hn[o * R + c] = acc2;
                }
                Rn[o] = r_s[e];
            }
        }
#pragma unroll
        for (int u = 0; u < (D + 127) / 128; ++u) {
            const int q = threadIdx.x + 128 * u;
            if (q < D) Gm[(size_t)k * D + q] = g[u];
        }
    }
}

// Columns: G^{L+2}(j) = sum r conj(h_{L+1}).
template <typename T, int R>
__global__ void __launch_bounds__(256)
k_grad_cols(const typename cvec<T>::type* __restrict__ H, const typename cvec<T>::type* __restrict__ Rc,
            const int32_t* __restrict__ seg, int nfib, double2* __restrict__ GL)
{
    typedef typename cvec<T>::type V;
    const int lane = threadIdx.x & 31;
    const int f = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (f >= nfib) return;
    const int s0 = seg[f], s1 = seg[f + 1];
    double2 g[R];
#pragma unroll
    for (int c = 0; c < R; ++c) g[c] = make_double2(0.0, 0.0);
    for (int p = s0 + lane; p < s1; p += 32) {
        const V rr = Rc[p];
#pragma unroll
        for (int c = 0; c < R; ++c) {
            const V h = H[(size_t)p * R + c];
            g[c].x += (double)rr.x * (double)h.x + (double)rr.y * (double)h.y;
            g[c].y += (double)rr.y * (double)h.x - (double)rr.x * (double)h.y;
        }
    }
#pragma unroll
    for (int c = 0; c < R; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            g[c].x += __shfl_xor_sync(0xffffffffu, g[c].x, o);
            g[c].y += __shfl_xor_sync(0xffffffffu, g[c].y, o);
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < R; ++c) GL[(size_t)f * R + c] = g[c];
    }
}

}  // namespace bfc
