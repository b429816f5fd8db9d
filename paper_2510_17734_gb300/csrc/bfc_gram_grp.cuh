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
// Two kernels: k_group_sums forms one record [s | M | v] per group (s the
// shared vector, M and v the sums of the other side); k_mid_gram_grp streams
// a slice's records through shared memory and accumulates the Kronecker
// updates.  Layout: the level order keeps each group contiguous; gseg[k] is
// the first group of slice k, gstart[g] the first position of group g.  Work
// per slice as in k_mid_gram: 4 x 4 complex tiles of the lower triangle of K
// owned by threads (tile I, J: rows a = 4I / R, c = 4I mod R + u; columns
// likewise).  Precision form: a group's term can be a large part of the
// slice's sum (16 row groups at the first level), so every term is added
// with Kahan compensation, and the group sums are compensated across blocks
// of 16 entries; the error of K then matches the per-entry kernels' (the
// rounding of the stored complex64 record dominates both).  Same output
// record as k_mid_gram.
#pragma once

#include "bfc_kernels.cuh"

namespace bfc {

template <typename V> __device__ __forceinline__ V make_conj(V a)
{
    a.y = -a.y;
    return a;
}

// 16-byte asynchronous global -> shared copy (L2 only) and its group waits.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem_src) : "memory");
}
template <int N> __device__ __forceinline__ void cp_async_wait_n()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem_src) : "memory");
}

// Group record [s | M | v] of rank R in values of type V: s at 0, M[c][c']
// at R + grp_m(c, c'), v at VOFF.  The rows c >= R/2 of M sit 64 bytes
// further on, so the 4 x 4 blocks of M the Gram tiles read at once (rows
// 0..3 and 4..7, column blocks 0 and 4) fall into distinct shared-memory
// banks.
template <typename V, int R> struct GrpRec {
    static constexpr int PAD = (int)(64 / sizeof(V));
    static constexpr int VOFF = R + R * R + PAD;
    static constexpr int RS = VOFF + R;
    __host__ __device__ static constexpr int m(int c, int cc) { return R + c * R + cc + (c >= R / 2 ? PAD : 0); }
};

// Shared-memory budget of k_group_sums: a block's entries (rows of the
// summed side and values) are staged when they fit.  CAP is the most a block
// stages (SMEM bytes); a launch sizes its dynamic shared memory for the
// level's largest block, at most CAP entries, so levels with small groups
// keep more blocks resident.
template <typename T, int R> struct GsumCfg {
    static constexpr int NTH = 128;
    static constexpr int GB = NTH / R;                    // groups per block
    static constexpr size_t VS = sizeof(typename cvec<T>::type);
    static constexpr int CAP = (int)(46080 / ((R + 1) * VS));   // staged entries per block
    static constexpr size_t SMEM = (size_t)CAP * (R + 1) * VS;
};

// Group sums of one middle level, one thread per (group, row a): the shared
// vector s of the group (h of a row group, w of a column group, taken from
// its first entry), and over the group's entries the sums
//   M[a][a'] = sum_e conj(u_e[a]) u_e[a'],   v[a] = sum_e conj(u_e[a]) t_e
// of the other environment u (w, resp. h).  Record per group, compute type:
// [s (R) | M (R x R, row-major) | v (R)].  A block's groups are contiguous
// in the level order, and so are their entries: when they fit (cap <= CAP
// entries, the dynamic shared memory of the launch, sized for the level's
// largest block), the rows u_e and values t_e of all of them are copied to
// shared memory at once (cp.async), so their loads overlap; otherwise they
// are read from global memory.  In the precision form the sums run in complex64 over blocks of 16
// entries, Kahan-compensated across blocks.
template <typename T, int R>
__global__ void __launch_bounds__(GsumCfg<T, R>::NTH)
k_group_sums(const typename cvec<T>::type* __restrict__ H, const typename cvec<T>::type* __restrict__ Wm,
             const typename cvec<T>::type* __restrict__ tv, const int32_t* __restrict__ gstart, int G, int by_col,
             typename cvec<T>::type* __restrict__ out, int cap)
{
    typedef typename cvec<T>::type V;
    typedef GsumCfg<T, R> C;
    typedef GrpRec<V, R> RL;
    constexpr int RS = RL::RS;
    extern __shared__ __align__(16) unsigned char smem[];
    V* su = (V*)smem;                          // [cap][R] rows
    V* st = su + (size_t)cap * R;              // [cap] values
    const V* Sv = by_col ? Wm : H;
    const V* Uv = by_col ? H : Wm;

    const int gb0 = blockIdx.x * C::GB;
    const int gb1 = min(gb0 + C::GB, G);
    const int E0 = gstart[gb0], E1 = gstart[gb1];
    const bool staged = E1 - E0 <= cap;
    if (staged) {
        // rows: (E1 - E0) R values, 16-byte pieces (a row is R * VS >= 32 bytes)
        const int rpieces = (int)((size_t)(E1 - E0) * R * C::VS / 16);
        const unsigned char* usrc = (const unsigned char*)(Uv + (size_t)E0 * R);
        for (int q = threadIdx.x; q < rpieces; q += C::NTH)
            cp_async16((unsigned char*)su + 16 * (size_t)q, usrc + 16 * (size_t)q);
        // values: one copy per entry (8 or 16 bytes)
        for (int q = threadIdx.x; q < E1 - E0; q += C::NTH) {
            if constexpr (sizeof(V) == 16)
                cp_async16(st + q, tv + E0 + q);
            else
                cp_async8(st + q, tv + E0 + q);
        }
        cp_async_commit();
        cp_async_wait_all();
    }
    __syncthreads();
    const int g = gb0 + (int)threadIdx.x / R, a = (int)threadIdx.x % R;
    if (g >= gb1) return;
    const int e0 = gstart[g], e1 = gstart[g + 1];
    // the block's entries in shared memory (staged) or global memory, indexed
    // from the block's first entry E0
    const V* ub = staged ? su : Uv + (size_t)E0 * R;
    const V* tb = staged ? st : tv + E0;
    V* o = out + (size_t)g * RS;
    o[a] = Sv[(size_t)e0 * R + a];
    V ms[R], vs;
    float mc[R][2], vc[2];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        ms[q] = czero<V>();
        mc[q][0] = mc[q][1] = 0.f;
    }
    vs = czero<V>();
    vc[0] = vc[1] = 0.f;
    for (int eb = e0; eb < e1; eb += 16) {
        V mp[R], vp = czero<V>();
#pragma unroll
        for (int q = 0; q < R; ++q) mp[q] = czero<V>();
        const int ee = min(eb + 16, e1);
        for (int e = eb; e < ee; ++e) {
            V u[R];
            const V* row = ub + (size_t)(e - E0) * R;
#pragma unroll
            for (int q = 0; q < R; ++q) u[q] = row[q];
            const V ua = row[a];   // one more load instead of a select chain
#pragma unroll
            for (int q = 0; q < R; ++q) cmacc(mp[q], ua, u[q]);
            cmacc(vp, ua, tb[e - E0]);
        }
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                kahan(ms[q].x, mc[q][0], mp[q].x);
                kahan(ms[q].y, mc[q][1], mp[q].y);
            }
            kahan(vs.x, vc[0], vp.x);
            kahan(vs.y, vc[1], vp.y);
        } else {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                ms[q].x += mp[q].x;
                ms[q].y += mp[q].y;
            }
            vs.x += vp.x;
            vs.y += vp.y;
        }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
        V m = ms[q];
        if constexpr (sizeof(T) == 4) {
            m.x -= mc[q][0];
            m.y -= mc[q][1];
        }
        o[RL::m(a, q)] = m;
    }
    if constexpr (sizeof(T) == 4) {
        vs.x -= vc[0];
        vs.y -= vc[1];
    }
    o[RL::VOFF + a] = vs;
}

// acc += x * y.  Precision form: (s, c) is a Kahan pair per component and
// the product enters with one rounding per component (the carried
// compensation is subtracted inside the fused multiply-adds); FP64: plain
// fused multiply-adds.
__device__ __forceinline__ void grp_acc(float2& s, float2& c, float2 x, float2 y)
{
    const float yr = __fmaf_rn(x.x, y.x, __fmaf_rn(-x.y, y.y, -c.x));
    const float yi = __fmaf_rn(x.x, y.y, __fmaf_rn(x.y, y.x, -c.y));
    float t = __fadd_rn(s.x, yr);
    c.x = __fsub_rn(__fsub_rn(t, s.x), yr);
    s.x = t;
    t = __fadd_rn(s.y, yi);
    c.y = __fsub_rn(__fsub_rn(t, s.y), yi);
    s.y = t;
}
__device__ __forceinline__ void grp_acc(double2& s, double2&, double2 x, double2 y) { cmac(s, x, y); }

// Packed (re, im) pairs of FP32 values and the f32x2 arithmetic of sm_100
// and later: one instruction acts on both components.
__device__ __forceinline__ uint64_t g2pack(float a, float b)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 g2unpack(uint64_t r)
{
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ uint64_t g2fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t g2add(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t g2sub(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// (s, nc) += x y with packed operands: X1 = (x.re, x.re), X2 = (x.im, x.im),
// Y = (y.re, y.im), Yr = i y = (-y.im, y.re), so x y = X1 Y + X2 Yr.  s is
// the Kahan sum and nc its negated compensation (the value is s + nc); the
// compensation enters inside the fused multiply-adds.
__device__ __forceinline__ void grp_acc2(uint64_t& s, uint64_t& nc, uint64_t X1, uint64_t X2, uint64_t Y,
                                         uint64_t Yr)
{
    const uint64_t q = g2fma(X1, Y, g2fma(X2, Yr, nc));   // x y - c
    const uint64_t t = g2add(s, q);
    nc = g2sub(q, g2sub(t, s));
    s = t;
}

template <typename T, int R> struct GrpCfg {
    static_assert(R == 4 || R == 8, "grouped Gram tiles need R in {4, 8}");
    static constexpr int D = R * R;
    static constexpr int NB = D / 4;
    static constexpr int NT = NB * (NB + 1) / 2;           // 4 x 4 tiles of the lower triangle
    static constexpr int CG = sizeof(T) == 4 ? 32 : 16;    // groups per chunk
    static constexpr int GT = (160 / NT) < 1 ? 1 : (160 / NT);
    static constexpr int G = GT > CG ? CG : GT;            // thread groups over the chunk's groups
    static constexpr int NW = NT * G;                      // tile threads
    static constexpr int NTH = ((NW + 31) / 32) * 32;
    // the right-hand side on the threads past the tiles when there are
    // enough of them (R = 8: 24 threads, 3 entries of y each), else on the
    // diagonal tiles
    static constexpr int NY = NTH - NW;
    static constexpr bool YSPARE = NY >= 8;
    static constexpr int YPT = YSPARE ? (D + NY - 1) / NY : 0;
    static constexpr int NST = 3;                          // ring stages
    static constexpr int NPK = D * (D + 1) / 2;
    typedef GrpRec<typename cvec<T>::type, R> RL;
    static constexpr int RS = RL::RS;                      // group record [s | M | v]
    static constexpr size_t VS = sizeof(typename cvec<T>::type);
    static constexpr int PIECES = (int)(RS * VS / 16);     // 16-byte pieces per record
    static_assert(RS * VS % 16 == 0, "records must be whole 16-byte pieces");
    static constexpr size_t STAGE = (size_t)CG * RS * VS;
    static constexpr size_t RING = NST * STAGE;
    static constexpr size_t KBYTES = G > 1 ? (size_t)(NPK + D) * sizeof(double2) : 0;
    static constexpr size_t SMEM = RING + KBYTES;
    static constexpr int MINB = sizeof(T) == 4 ? 3 : 2;
};

// Per-slice normal equations from the group records of k_group_sums (one
// block per slice, grid-stride).  Chunks of CG records stream through an
// NST-stage shared-memory ring by 16-byte cp.async copies; per group, the
// shared side's outer product is formed in registers (conj(s_a) s_a' for row
// groups; conj(s_c) s_c' for column groups) and multiplied with the other
// side's sums M, each product added to the tile's accumulators (compensated
// per group in the precision form: a group's term can be a large part of
// the slice's sum).
template <typename T, int R, int BY_COL>
__global__ void __launch_bounds__(GrpCfg<T, R>::NTH, GrpCfg<T, R>::MINB)
k_mid_gram_grp(const typename cvec<T>::type* __restrict__ grec, const int32_t* __restrict__ gseg,
               typename cvec<T>::type* __restrict__ rec, int S)
{
    typedef typename cvec<T>::type V;
    typedef GrpCfg<T, R> C;
    constexpr int D = C::D, NPK = C::NPK, CG = C::CG, NTH = C::NTH, RS = C::RS, NST = C::NST;
    extern __shared__ __align__(16) unsigned char smem[];
    typedef typename C::RL RL;
    V* ring = (V*)smem;                           // [NST][CG][RS]
    double2* Kacc = (double2*)(smem + C::RING);   // thread-group reduction (G > 1)

    const int tid = threadIdx.x;
    const bool worker = tid < C::NW;
    const bool ythread = C::YSPARE && !worker;
    const int grp = worker ? tid / C::NT : 0, tile = worker ? tid - grp * C::NT : 0;
    int I = 0;
    while ((I + 1) * (I + 2) / 2 <= tile) ++I;
    const int J = tile - I * (I + 1) / 2;
    const bool diag = !C::YSPARE && (I == J);
    // row p = 4 I + u of K is the pair (a, c) = (p / R, p mod R): a = aI, c = cI + u
    const int aI = (4 * I) / R, cI = (4 * I) % R, aJ = (4 * J) / R, cJ = (4 * J) % R;
    // right-hand side entries p = yb + NY x of a spare thread
    const int yb = tid - C::NW;

    // records [gfirst, gfirst + cnt) into ring stage st
    auto issue = [&](int st, int gfirst, int cnt) {
        const unsigned char* src = (const unsigned char*)(grec + (size_t)gfirst * RS);
        unsigned char* dst = (unsigned char*)(ring + (size_t)st * CG * RS);
        const int pieces = cnt * C::PIECES;
        for (int q = tid; q < pieces; q += NTH) cp_async16(dst + 16 * (size_t)q, src + 16 * (size_t)q);
    };

    for (int k = blockIdx.x; k < S; k += gridDim.x) {
        const int g0 = gseg[k], g1 = gseg[k + 1];
        const int nch = (g1 - g0 + CG - 1) / CG;
        // tiles: s_/c_ (Kahan pairs); right-hand side: ys/yc (diagonal tiles
        // or spare threads)
        V s_[4][4], c_[4][4], ys[4], yc[4];
        uint64_t s2[4][4], n2[4][4];   // complex64 tiles: packed Kahan sums, negated compensations
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            ys[u] = czero<V>();
            yc[u] = czero<V>();
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                s_[u][v] = czero<V>();
                c_[u][v] = czero<V>();
                s2[u][v] = 0ull;
                n2[u][v] = 0ull;
            }
        }
        __syncthreads();  // previous slice done with the ring and Kacc
#pragma unroll
        for (int c = 0; c < NST - 1; ++c) {
            if (c < nch) issue(c, g0 + c * CG, min(CG, g1 - g0 - c * CG));
            cp_async_commit();
        }
        for (int c = 0; c < nch; ++c) {
            cp_async_wait_n<NST - 2>();   // this thread's copies of chunk c landed
            __syncthreads();              // everyone's; stage (c - 1) mod NST is free
            const int cn = c + NST - 1;
            if (cn < nch) issue(cn % NST, g0 + cn * CG, min(CG, g1 - g0 - cn * CG));
            cp_async_commit();
            const V* buf = ring + (size_t)(c % NST) * CG * RS;
            const int cnt = min(CG, g1 - g0 - c * CG);
            if constexpr (sizeof(T) == 4) {
              if (worker) {
                for (int gi = grp; gi < cnt; gi += C::G) {
                    const V* gr = buf + gi * RS;
                    if constexpr (!BY_COL) {
                        // X = conj(h) h^T from s = h; Y = M (sums of the w side)
                        const V x = cmul(make_conj(gr[aI]), gr[aJ]);
                        const uint64_t X1 = g2pack(x.x, x.x), X2 = g2pack(x.y, x.y);
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            V yr[4];
                            load4(yr, gr + RL::m(cI + u, cJ));
#pragma unroll
                            for (int v = 0; v < 4; ++v)
                                grp_acc2(s2[u][v], n2[u][v], X1, X2, g2pack(yr[v].x, yr[v].y),
                                         g2pack(-yr[v].y, yr[v].x));
                        }
                        if (diag) {
                            const V xv = make_conj(gr[aI]);
#pragma unroll
                            for (int u = 0; u < 4; ++u) grp_acc(ys[u], yc[u], xv, gr[RL::VOFF + cI + u]);
                        }
                    } else {
                        // X = M (sums of the h side); Y = conj(w) w^T from s = w:
                        // term (u, v) = (conj(s_cI+u) x) s_cJ+v
                        const V x = gr[RL::m(aI, aJ)];
                        V sj[4], si[4];
                        load4(sj, gr + cJ);
                        load4(si, gr + cI);
                        uint64_t Y[4], Q[4];
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            Y[v] = g2pack(sj[v].x, sj[v].y);
                            Q[v] = g2pack(-sj[v].y, sj[v].x);
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const V xa = cmul(make_conj(si[u]), x);
                            const uint64_t X1 = g2pack(xa.x, xa.x), X2 = g2pack(xa.y, xa.y);
#pragma unroll
                            for (int v = 0; v < 4; ++v) grp_acc2(s2[u][v], n2[u][v], X1, X2, Y[v], Q[v]);
                        }
                        if (diag) {
                            const V xv = gr[RL::VOFF + aI];
#pragma unroll
                            for (int u = 0; u < 4; ++u) grp_acc(ys[u], yc[u], xv, make_conj(si[u]));
                        }
                    }
                }
              }
            } else if (worker) {
                for (int gi = grp; gi < cnt; gi += C::G) {
                    const V* gr = buf + gi * RS;
                    if constexpr (!BY_COL) {
                        // X = conj(h) h^T from s = h; Y = M (sums of the w side)
                        const V x = cmul(make_conj(gr[aI]), gr[aJ]);
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            V yr[4];
                            load4(yr, gr + RL::m(cI + u, cJ));
#pragma unroll
                            for (int v = 0; v < 4; ++v) grp_acc(s_[u][v], c_[u][v], x, yr[v]);
                        }
                        if (diag) {
                            const V xv = make_conj(gr[aI]);
#pragma unroll
                            for (int u = 0; u < 4; ++u) grp_acc(ys[u], yc[u], xv, gr[RL::VOFF + cI + u]);
                        }
                    } else {
                        // X = M (sums of the h side); Y = conj(w) w^T from s = w
                        const V x = gr[RL::m(aI, aJ)];
                        V sj[4], si[4];
                        load4(sj, gr + cJ);
                        load4(si, gr + cI);
#pragma unroll
                        for (int v = 0; v < 4; ++v) sj[v] = cmul(x, sj[v]);
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const V a = make_conj(si[u]);
#pragma unroll
                            for (int v = 0; v < 4; ++v) grp_acc(s_[u][v], c_[u][v], a, sj[v]);
                        }
                        if (diag) {
                            const V xv = gr[RL::VOFF + aI];
#pragma unroll
                            for (int u = 0; u < 4; ++u) grp_acc(ys[u], yc[u], xv, make_conj(si[u]));
                        }
                    }
                }
            }
            if (ythread) {
                // y[(a, c)] += xv[a] yv[c] for p = yb + NY x
                for (int gi = 0; gi < cnt; ++gi) {
                    const V* gr = buf + gi * RS;
#pragma unroll
                    for (int x = 0; x < C::YPT; ++x) {
                        const int p = yb + C::NY * x;
                        if (p < D) {
                            const int a = p / R, cc = p - (p / R) * R;
                            const V xv = BY_COL ? gr[RL::VOFF + a] : make_conj(gr[a]);
                            const V yv = BY_COL ? make_conj(gr[cc]) : gr[RL::VOFF + cc];
                            grp_acc(ys[x], yc[x], xv, yv);
                        }
                    }
                }
            }
        }
        cp_async_wait_n<0>();
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float2 t = g2unpack(g2add(s2[u][v], n2[u][v]));
                    s_[u][v].x = t.x;
                    s_[u][v].y = t.y;
                }
                ys[u].x = __fsub_rn(ys[u].x, yc[u].x);
                ys[u].y = __fsub_rn(ys[u].y, yc[u].y);
            }
        }
        V* out = rec + (size_t)k * (NPK + D);
        if constexpr (C::G == 1) {
            if (worker) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int p = I * 4 + u;
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int q = J * 4 + v;
                        if (q <= p) out[tri(p, q)] = s_[u][v];
                    }
                    if (diag) out[NPK + p] = ys[u];
                }
            } else if (ythread) {
#pragma unroll
                for (int x = 0; x < C::YPT; ++x) {
                    const int p = yb + C::NY * x;
                    if (p < D) out[NPK + p] = ys[x];
                }
            }
        } else {
            static_assert(C::G == 1 || !C::YSPARE, "the thread-group reduction takes y from the diagonal tiles");
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
                                Kacc[tri(p, q)].x += (double)s_[u][v].x;
                                Kacc[tri(p, q)].y += (double)s_[u][v].y;
                            }
                        }
                        if (diag) {
                            Kacc[NPK + p].x += (double)ys[u].x;
                            Kacc[NPK + p].y += (double)ys[u].y;
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
