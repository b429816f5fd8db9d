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

// Four consecutive complex values from 16-byte-aligned shared memory.
__device__ __forceinline__ void load4(float2 (&d)[4], const float2* p)
{
    const float4 a = *reinterpret_cast<const float4*>(p);
    const float4 b = *reinterpret_cast<const float4*>(p + 2);
    d[0] = make_float2(a.x, a.y);
    d[1] = make_float2(a.z, a.w);
    d[2] = make_float2(b.x, b.y);
    d[3] = make_float2(b.z, b.w);
}
__device__ __forceinline__ void load4(double2 (&d)[4], const double2* p)
{
#pragma unroll
    for (int u = 0; u < 4; ++u) d[u] = p[u];
}

// Slice id of the middle factor S^{m+1}: psi^{-1}(i_0..i_{L-m}, j_0..j_{m-1}).
__device__ __forceinline__ int slice_of(int pi, int pj, int m, int L)
{
    return ((pi >> (m - 1)) << m) | (pj >> (L - m));
}

// Packed lower-triangular index (p >= q).
__host__ __device__ __forceinline__ constexpr int tri(int p, int q) { return (p * (p + 1) >> 1) + q; }

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
// Normal equations of Alg. 1 (complex form): for a block (one fiber of S^1 or
// S^{L+2}, or one slice of a middle factor) with design vectors a_e,
//   K = sum conj(a_e) a_e^T + lambda I,   y = sum conj(a_e) t_e,   K s = y.
// Every kernel that accumulates K and y writes them, packed lower-triangular
// (element (p, q), p >= q, at tri(p, q)) followed by y, to a per-block
// record; a solve kernel then factors and solves.
//
// FP64 on this GPU runs at 1/64 of the FP32 rate and a warp-wide FP64
// instruction holds an SM sub-partition's FP64 pipe for tens of cycles
// whatever the number of active lanes, so every FP64 stage below keeps all 32
// lanes busy: small systems are solved one per thread, large ones with rows
// spread over the lanes.

template <typename E> __device__ __forceinline__ void csub_mul_conj(E& acc, E a, E b)
{
    // acc -= a * conj(b)
    acc.x -= a.x * b.x + a.y * b.y;
    acc.y -= a.y * b.x - a.x * b.y;
}

// Hermitian Cholesky + two triangular solves for one small system held by one
// thread (R compile-time: the loops unroll and K, y stay in registers).
// K: packed lower (R(R+1)/2), y: right-hand side, overwritten by the solution.
template <int R>
__device__ __forceinline__ bool thread_chol_solve(double2 (&K)[R * (R + 1) / 2], double2 (&y)[R], double tol)
{
#pragma unroll
    for (int c = 0; c < R; ++c) {
        double d = K[tri(c, c)].x;
#pragma unroll
        for (int q = 0; q < c; ++q) d -= K[tri(c, q)].x * K[tri(c, q)].x + K[tri(c, q)].y * K[tri(c, q)].y;
        if (!(d > tol)) return false;
        const double piv = sqrt(d), inv = 1.0 / piv;
        K[tri(c, c)] = make_double2(piv, inv);  // .y keeps 1/piv for the solves
#pragma unroll
        for (int row = c + 1; row < R; ++row) {
            double2 acc = K[tri(row, c)];
#pragma unroll
            for (int q = 0; q < c; ++q) csub_mul_conj(acc, K[tri(row, q)], K[tri(c, q)]);
            K[tri(row, c)] = make_double2(acc.x * inv, acc.y * inv);
        }
    }
#pragma unroll
    for (int row = 0; row < R; ++row) {
        double2 acc = y[row];
#pragma unroll
        for (int q = 0; q < row; ++q) {
            const double2 l = K[tri(row, q)], z = y[q];
            acc.x -= l.x * z.x - l.y * z.y;
            acc.y -= l.x * z.y + l.y * z.x;
        }
        const double inv = K[tri(row, row)].y;
        y[row] = make_double2(acc.x * inv, acc.y * inv);
    }
#pragma unroll
    for (int row = R - 1; row >= 0; --row) {
        double2 acc = y[row];
#pragma unroll
        for (int q = row + 1; q < R; ++q) {
            const double2 l = K[tri(q, row)], z = y[q];
            acc.x -= l.x * z.x + l.y * z.y;
            acc.y -= l.x * z.y - l.y * z.x;
        }
        const double inv = K[tri(row, row)].y;
        y[row] = make_double2(acc.x * inv, acc.y * inv);
    }
    return true;
}

// ------------------------------------------------------------------------
// Outer fibers, stage 1: one warp per fiber accumulates K and y (r x r) over
// the fiber's entries.  A: design vectors in the level order (w_0 for the S^1
// rows, h_{L+1} for the S^{L+2} columns).  Lanes own the R(R+1)/2 + R items;
// in float the per-chunk partials are folded into Kahan-compensated sums.
// Output record per fiber: [K packed (R(R+1)/2) | y (R)] in FP64.
template <typename T, int R>
__global__ void __launch_bounds__(128)
k_outer_gram(const typename cvec<T>::type* __restrict__ A, const typename cvec<T>::type* __restrict__ tv,
             const int32_t* __restrict__ seg, int nfib, double2* __restrict__ rec)
{
    typedef typename cvec<T>::type V;
    constexpr bool COMP = sizeof(T) == 4;
    constexpr int NP = R * (R + 1) / 2;
    constexpr int NI = NP + R;
    constexpr int IPL = (NI + 31) / 32;
    constexpr int WPB = 4;
    __shared__ V a_s[WPB][32 * R];
    __shared__ V t_s[WPB][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int f = blockIdx.x * WPB + wib;
    if (f >= nfib) return;  // whole warp leaves; only warp-level barriers below
    const int s0 = seg[f], s1 = seg[f + 1];

    int ip[IPL], iq[IPL];
#pragma unroll
    for (int u = 0; u < IPL; ++u) {
        const int it = lane + 32 * u;
        ip[u] = -1;
        iq[u] = -1;
        if (it < NP) {
            int p = 0;
            while ((p + 1) * (p + 2) / 2 <= it) ++p;
            ip[u] = p;
            iq[u] = it - p * (p + 1) / 2;
        } else if (it < NI) {
            ip[u] = it - NP;
            iq[u] = -2;  // right-hand side item
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
#pragma unroll
    for (int u = 0; u < IPL; ++u) {
        const int it = lane + 32 * u;
        if (it < NI) {
            const double2 v = COMP ? make_double2((double)sum[u].x - (double)cmp[u].x,
                                                  (double)sum[u].y - (double)cmp[u].y)
                                   : to_d2(acc[u]);
            rec[(size_t)f * NI + it] = v;
        }
    }
}

// Outer fibers, stage 2: one thread per fiber solves K + lambda I in FP64
// (32 independent fibers per warp keep every lane of the FP64 pipe busy).
// A system whose pivot falls to <= tol keeps its old fiber and is counted.
template <typename T, int R>
__global__ void __launch_bounds__(64)
k_outer_solve(const double2* __restrict__ rec, int nfib, double lambda, double ridge, double2* __restrict__ zd,
              typename cvec<T>::type* __restrict__ zt, unsigned long long* __restrict__ nsing)
{
    typedef typename cvec<T>::type V;
    constexpr int NP = R * (R + 1) / 2;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfib) return;
    double2 K[NP], y[R];
    const double2* src = rec + (size_t)f * (NP + R);
#pragma unroll
    for (int q = 0; q < NP; ++q) K[q] = src[q];
#pragma unroll
    for (int q = 0; q < R; ++q) y[q] = src[NP + q];
    double tr0 = 0.0;
#pragma unroll
    for (int p = 0; p < R; ++p) tr0 += K[tri(p, p)].x;
    const double lam = fmax(lambda, ridge * tr0 / R);
#pragma unroll
    for (int p = 0; p < R; ++p) K[tri(p, p)].x += lam;
    const double tol = lam > 0.0 ? 0.0 : 1e-14 * (tr0 + R * lam);
    if (thread_chol_solve<R>(K, y, tol)) {
#pragma unroll
        for (int c = 0; c < R; ++c) {
            zd[(size_t)f * R + c] = y[c];
            zt[(size_t)f * R + c] = from_d2<V>(y[c]);
        }
    } else {
        atomicAdd(nsing, 1ull);
    }
}

// Outer fibers, stage 3 (one warp per fiber).  Rows (S^1): h_1 = z1(i, :) for
// every entry, written into order 1.  Columns (S^{L+2}): x = h_{L+1}^T zL(j),
// per-fiber sums of |t - x|^2 and |t|^2 for the training error.
template <typename T, int R, bool COLS>
__global__ void __launch_bounds__(128)
k_outer_post(const typename cvec<T>::type* __restrict__ A, const typename cvec<T>::type* __restrict__ tv,
             const int32_t* __restrict__ seg, int nfib, const typename cvec<T>::type* __restrict__ zt,
             const int32_t* __restrict__ nxt, typename cvec<T>::type* __restrict__ Hn,
             double* __restrict__ err_part)
{
    typedef typename cvec<T>::type V;
    const int lane = threadIdx.x & 31;
    const int f = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (f >= nfib) return;
    const int s0 = seg[f], s1 = seg[f + 1];
    V zf[R];
#pragma unroll
    for (int c = 0; c < R; ++c) zf[c] = zt[(size_t)f * R + c];
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
            const V t = tv[p];
            const double dx = (double)t.x - (double)x.x, dy = (double)t.y - (double)x.y;
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
// Middle level m, stage 1 (Gram): one CTA per slice k of S^{m+1}.
//   a_e = h_m(e) (x) w_m(e), a[p r + c] = h_p w_c, K = sum conj(a) a^T,
//   y = sum conj(a) t over the slice's entries (Alg. 1 middle branch).
// Threads own 4x4 complex tiles of the lower triangle of K; entries are
// staged in shared memory in chunks of CE and split over G thread groups.  In
// float every chunk partial (registers) is folded into a Kahan-compensated
// running sum (sum in registers, compensation in shared memory, so several
// CTAs fit on one SM).  Output record per slice: [K packed | y] in the compute
// type (the compensated sums rounded once).
template <typename T, int R> struct GramCfg {
    static constexpr int D = R * R;
    static constexpr int DP = (D + 3) / 4 * 4;
    static constexpr int NB = DP / 4;
    static constexpr int NT = NB * (NB + 1) / 2;
    static constexpr int CE = (DP <= 64) ? 64 : 32;
    static constexpr int GT = (160 / NT) < 1 ? 1 : (160 / NT);
    static constexpr int G = GT > CE ? CE : GT;
    static constexpr int NTH = ((NT * G + 31) / 32) * 32;
    static constexpr bool COMP = sizeof(T) == 4;
    static constexpr int NPK = D * (D + 1) / 2;
    static constexpr int CSTRIDE = 40;  // compensation floats per worker thread
    static constexpr size_t VS = sizeof(typename cvec<T>::type);
    static constexpr size_t CBYTES = COMP ? (size_t)NTH * CSTRIDE * sizeof(float) : 0;
    static constexpr size_t KBYTES = G > 1 ? (size_t)(NPK + D) * sizeof(double2) : 0;
    static constexpr size_t UBYTES = ((CBYTES > KBYTES ? CBYTES : KBYTES) + 15) / 16 * 16;
    static constexpr size_t SMEM = 2 * (size_t)CE * R * VS + (size_t)CE * DP * VS + (size_t)CE * VS + UBYTES + 16;
};

template <typename T, int R>
__global__ void __launch_bounds__(GramCfg<T, R>::NTH)
k_mid_gram(const typename cvec<T>::type* __restrict__ H, const typename cvec<T>::type* __restrict__ Wm,
           const typename cvec<T>::type* __restrict__ tv, const int32_t* __restrict__ seg,
           typename cvec<T>::type* __restrict__ rec, int S)
{
    typedef typename cvec<T>::type V;
    typedef GramCfg<T, R> C;
    constexpr int D = C::D, DP = C::DP, NPK = C::NPK;
    extern __shared__ __align__(16) unsigned char smem[];
    V* h_s = (V*)smem;
    V* w_s = h_s + C::CE * R;
    V* a_s = w_s + C::CE * R;
    V* t_s = a_s + C::CE * DP;
    unsigned char* U = (unsigned char*)(t_s + C::CE);
    float* c_s = (float*)U;
    double2* Kacc = (double2*)U;

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
            for (int q = tid; q < cnt * R; q += nth) {
                h_s[q] = H[(size_t)base * R + q];
                w_s[q] = Wm[(size_t)base * R + q];
            }
            for (int e = tid; e < cnt; e += nth) t_s[e] = tv[base + e];
            __syncthreads();
            for (int idx = tid; idx < cnt * DP; idx += nth) {
                const int e = idx / DP, q = idx - e * DP;
                V a = czero<V>();
                if (q < D) {
                    const int pa = q / R, pc = q - pa * R;
                    a = cmul(h_s[e * R + pa], w_s[e * R + pc]);
                }
                a_s[idx] = a;
            }
            __syncthreads();
            if (worker) {
                for (int e = grp; e < cnt; e += C::G) {
                    const V* ae = a_s + e * DP;
                    V ap[4], aq[4];
                    load4(ap, ae + I * 4);
                    load4(aq, ae + J * 4);
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
                            float& cx = c_s[(2 * (u * 4 + v)) * C::NTH + tid];
                            float& cy = c_s[(2 * (u * 4 + v) + 1) * C::NTH + tid];
                            kahan(sx, cx, (float)acc[u][v].x);
                            kahan(sy, cy, (float)acc[u][v].y);
                            sum[u][v].x = sx; sum[u][v].y = sy;
                            acc[u][v] = czero<V>();
                        }
                        if (diag) {
                            float sx = (float)ysum[u].x, sy = (float)ysum[u].y;
                            float& cx = c_s[(32 + 2 * u) * C::NTH + tid];
                            float& cy = c_s[(32 + 2 * u + 1) * C::NTH + tid];
                            kahan(sx, cx, (float)yacc[u].x);
                            kahan(sy, cy, (float)yacc[u].y);
                            ysum[u].x = sx; ysum[u].y = sy;
                            yacc[u] = czero<V>();
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (C::COMP && worker) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    acc[u][v].x = sum[u][v].x - c_s[(2 * (u * 4 + v)) * C::NTH + tid];
                    acc[u][v].y = sum[u][v].y - c_s[(2 * (u * 4 + v) + 1) * C::NTH + tid];
                }
                if (diag) {
                    yacc[u].x = ysum[u].x - c_s[(32 + 2 * u) * C::NTH + tid];
                    yacc[u].y = ysum[u].y - c_s[(32 + 2 * u + 1) * C::NTH + tid];
                }
            }
        }
        V* out = rec + (size_t)k * (NPK + D);
        if (C::G == 1) {
            if (worker) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int p = I * 4 + u;
                    if (p < D) {
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const int q = J * 4 + v;
                            if (q <= p) out[tri(p, q)] = acc[u][v];
                        }
                        if (diag) out[NPK + p] = yacc[u];
                    }
                }
            }
        } else {
            __syncthreads();  // compensation reads done before Kacc overwrites them
            for (int q = tid; q < NPK + D; q += nth) Kacc[q] = make_double2(0.0, 0.0);
            __syncthreads();
            for (int g = 0; g < C::G; ++g) {  // deterministic order over the groups
                if (worker && grp == g) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int p = I * 4 + u;
                        if (p < D) {
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
                }
                __syncthreads();
            }
            for (int q = tid; q < NPK + D; q += nth) out[q] = from_d2<V>(Kacc[q]);
        }
    }
}

// ------------------------------------------------------------------------
// Warp-level Hermitian Cholesky (K = L L^H) of a D x D packed lower matrix
// in shared or global memory.  Right-looking; the trailing update of each
// column is flattened over all (row, col) pairs so every lane has work.  The
// diagonal of L is real, so its imaginary slot stores 1 / L_cc for the
// triangular solves.  Returns false (warp-uniform) when a pivot is <= tol.
template <typename E, typename S>
__device__ bool warp_chol(E* Lm, int D, S tol, int lane)
{
    for (int c = 0; c < D; ++c) {
        __syncwarp();
        const S d = Lm[tri(c, c)].x;
        if (!(d > tol)) return false;
        const S piv = sqrt(d), inv = S(1) / piv;
        __syncwarp();
        if (lane == 0) {
            E v;
            v.x = piv;
            v.y = inv;  // the factor's diagonal is real: its imaginary slot keeps 1 / L_cc
            Lm[tri(c, c)] = v;
        }
        for (int row = c + 1 + lane; row < D; row += 32) {
            E l = Lm[tri(row, c)];
            l.x *= inv;
            l.y *= inv;
            Lm[tri(row, c)] = l;
        }
        __syncwarp();
        const int m = D - c - 1;
        const int npairs = m * (m + 1) / 2;
        int rr = 0, qq = lane;
        while (rr < m && qq > rr) { qq -= rr + 1; ++rr; }
        for (int idx = lane; idx < npairs; idx += 32) {
            const int r_ = c + 1 + rr, q_ = c + 1 + qq;
            const E a = Lm[tri(r_, c)], bq = Lm[tri(q_, c)];
            E cur = Lm[tri(r_, q_)];
            csub_mul_conj(cur, a, bq);
            Lm[tri(r_, q_)] = cur;
            qq += 32;
            while (rr < m && qq > rr) { qq -= rr + 1; ++rr; }
        }
    }
    __syncwarp();
    return true;
}

// Column-oriented triangular solves with the right-hand side spread over the
// lanes: row p lives in slot p / 32 of lane p % 32.  L z = b, then L^H x = z.
template <typename E, typename S, int NS>
__device__ __forceinline__ void warp_chol_solve(const E* Lm, int D, E (&bv)[NS], int lane)
{
#pragma unroll
    for (int slot = 0; slot < NS; ++slot) {
        for (int owner = 0; owner < 32; ++owner) {
            const int p = slot * 32 + owner;
            if (p >= D) break;
            E zp;
            zp.x = __shfl_sync(0xffffffffu, bv[slot].x, owner);
            zp.y = __shfl_sync(0xffffffffu, bv[slot].y, owner);
            const S inv = Lm[tri(p, p)].y;
            zp.x *= inv;
            zp.y *= inv;
            if (lane == owner) bv[slot] = zp;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int q = lane + 32 * s;
                if (q > p && q < D) {
                    const E l = Lm[tri(q, p)];
                    bv[s].x -= l.x * zp.x - l.y * zp.y;
                    bv[s].y -= l.x * zp.y + l.y * zp.x;
                }
            }
        }
    }
#pragma unroll
    for (int slot = NS - 1; slot >= 0; --slot) {
        for (int owner = 31; owner >= 0; --owner) {
            const int p = slot * 32 + owner;
            if (p >= D) continue;
            E xp;
            xp.x = __shfl_sync(0xffffffffu, bv[slot].x, owner);
            xp.y = __shfl_sync(0xffffffffu, bv[slot].y, owner);
            const S inv = Lm[tri(p, p)].y;
            xp.x *= inv;
            xp.y *= inv;
            if (lane == owner) bv[slot] = xp;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int q = lane + 32 * s;
                if (q < p) {
                    const E l = Lm[tri(p, q)];   // conj(l) * xp
                    bv[s].x -= l.x * xp.x + l.y * xp.y;
                    bv[s].y -= l.x * xp.y - l.y * xp.x;
                }
            }
        }
    }
}

template <typename T, int R> struct SolveCfg {
    static constexpr int D = R * R;
    static constexpr int NPK = D * (D + 1) / 2;
    static constexpr int NS = (D + 31) / 32;
    static constexpr bool MIXED = sizeof(T) == 4;
    // per warp: factor (compute type, padded to 16 bytes), FP64 solution
    // vector, new slice (compute type)
    static constexpr size_t LBYTES = ((size_t)NPK * sizeof(typename cvec<T>::type) + 15) / 16 * 16;
    static constexpr size_t WBYTES = (LBYTES + (size_t)D * sizeof(double2) +
                                      (size_t)D * sizeof(typename cvec<T>::type) + (size_t)D * sizeof(T) + 15) /
                                     16 * 16;
    static constexpr int WPB0 = (int)((96 * 1024) / WBYTES);
    static constexpr int WPB = WPB0 < 1 ? 1 : (WPB0 > 4 ? 4 : WPB0);
    static constexpr size_t SMEM = WBYTES * WPB;
};

// Middle level m, stage 2 (solve + left update): one warp per slice.
// Precision form (float): complex64 Cholesky of the Jacobi-equilibrated
// S (K + lambda I) S, complex64 solve, then up to three steps of FP64
// iterative refinement (residual y - (K + lambda I) s in FP64 with rows spread
// over the lanes, correction through the complex64 factor);
// if the factorization breaks down or the refinement does not contract, the
// system is solved by an FP64 Cholesky instead (counted in nref).  FP64 path
// (double): FP64 Cholesky directly.  The slice is written row-major in FP64
// and the compute type; then h_{m+1}(e) = h_m(e)^T Z^{m+1}(k) for the slice's
// entries is scattered into order m+1.  A singular system keeps its old slice.
template <typename T, int R>
__global__ void __launch_bounds__(32 * SolveCfg<T, R>::WPB)
k_mid_solve(const typename cvec<T>::type* __restrict__ rec, const typename cvec<T>::type* __restrict__ H,
            const int32_t* __restrict__ seg, const int32_t* __restrict__ nxt,
            typename cvec<T>::type* __restrict__ Hn, double2* __restrict__ Zd,
            typename cvec<T>::type* __restrict__ Zt, double2* __restrict__ fb, double lambda_in, double ridge,
            unsigned long long* __restrict__ nsing, unsigned long long* __restrict__ nref, int S)
{
    typedef typename cvec<T>::type V;
    typedef SolveCfg<T, R> C;
    constexpr int D = C::D, NPK = C::NPK, NS = C::NS;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char* base = smem + (size_t)wib * C::WBYTES;
    V* Lm = (V*)base;
    double2* s_d = (double2*)(base + C::LBYTES);
    V* zt_s = (V*)(s_d + D);
    T* sc_s = (T*)(zt_s + D);  // Jacobi scaling of the complex64 factorization

    for (int k = blockIdx.x * C::WPB + wib; k < S; k += gridDim.x * C::WPB) {
        const V* K = rec + (size_t)k * (NPK + D);
        __syncwarp();
        double tr = 0.0;
        for (int p = lane; p < D; p += 32) tr += (double)K[tri(p, p)].x;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
        // lambda, raised to the ridge floor (relative to the mean diagonal) when set
        const double lambda = fmax(lambda_in, ridge * tr / D);
        const double tol = lambda > 0.0 ? 0.0 : 1e-14 * (tr + D * lambda);
        if constexpr (C::MIXED) {
            // equilibrate: factor S (K + lambda I) S with S = diag(K_pp + lambda)^(-1/2)
            for (int p = lane; p < D; p += 32) {
                const double dp = (double)K[tri(p, p)].x + lambda;
                sc_s[p] = dp > 0.0 ? (T)(1.0 / sqrt(dp)) : (T)1;
            }
            __syncwarp();
            int rr = 0, qq = lane;
            while (qq > rr) { qq -= rr + 1; ++rr; }
            for (int q = lane; q < NPK; q += 32) {
                V v = K[q];
                if (rr == qq) v.x += (T)lambda;
                const T f = sc_s[rr] * sc_s[qq];
                v.x *= f;
                v.y *= f;
                Lm[q] = v;
                qq += 32;
                while (qq > rr) { qq -= rr + 1; ++rr; }
            }
        } else {
            for (int q = lane; q < NPK; q += 32) Lm[q] = K[q];
            __syncwarp();
            for (int p = lane; p < D; p += 32) Lm[tri(p, p)].x += (T)lambda;
        }
        __syncwarp();
        double2 sv[NS];
        bool ok;
        if constexpr (C::MIXED) {
            bool conv = false;
            if (warp_chol<V, T>(Lm, D, (T)tol, lane)) {
                V bv[NS];
                T scl[NS];
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    const int p = lane + 32 * s;
                    scl[s] = p < D ? sc_s[p] : (T)0;
                    bv[s] = p < D ? K[NPK + p] : czero<V>();
                    bv[s].x *= scl[s];
                    bv[s].y *= scl[s];
                }
                warp_chol_solve<V, T, NS>(Lm, D, bv, lane);
#pragma unroll
                for (int s = 0; s < NS; ++s) sv[s] = make_double2((double)(bv[s].x * scl[s]), (double)(bv[s].y * scl[s]));
                // FP64 copy of K for the residuals (converted once per slice)
                double2* Kd = fb + (size_t)k * NPK;
                for (int q = lane; q < NPK; q += 32) Kd[q] = to_d2(K[q]);
                __syncwarp();
                double dmax = 0.0, smax = 0.0;
                for (int it = 0; it < 3; ++it) {
                    // FP64 residual r = y - (K + lambda I) s, rows over the lanes
                    __syncwarp();
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        const int p = lane + 32 * s;
                        if (p < D) s_d[p] = sv[s];
                    }
                    __syncwarp();
                    double2 rv[NS];
                    double rmax = 0.0;
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        const int p = lane + 32 * s;
                        double2 acc = make_double2(0.0, 0.0);
                        if (p < D) {
                            const double2 yp = to_d2(K[NPK + p]);
                            acc.x = yp.x - lambda * sv[s].x;
                            acc.y = yp.y - lambda * sv[s].y;
                            for (int q = 0; q <= p; ++q) {   // K_pq s_q
                                const double2 kk = Kd[tri(p, q)], sq = s_d[q];
                                acc.x -= kk.x * sq.x - kk.y * sq.y;
                                acc.y -= kk.x * sq.y + kk.y * sq.x;
                            }
                            for (int q = p + 1; q < D; ++q) {  // conj(K_qp) s_q
                                const double2 kk = Kd[tri(q, p)], sq = s_d[q];
                                acc.x -= kk.x * sq.x + kk.y * sq.y;
                                acc.y -= kk.x * sq.y - kk.y * sq.x;
                            }
                        }
                        rv[s] = acc;
                        rmax = fmax(rmax, fmax(fabs(acc.x), fabs(acc.y)));
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
                    const double sc = rmax > 0.0 ? rmax : 1.0;
                    const double isc = 1.0 / sc;
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        bv[s] = from_d2<V>(make_double2(rv[s].x * isc, rv[s].y * isc));
                        bv[s].x *= scl[s];
                        bv[s].y *= scl[s];
                    }
                    warp_chol_solve<V, T, NS>(Lm, D, bv, lane);
                    dmax = 0.0;
                    smax = 0.0;
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        const double dx = (double)(bv[s].x * scl[s]) * sc, dy = (double)(bv[s].y * scl[s]) * sc;
                        sv[s].x += dx;
                        sv[s].y += dy;
                        dmax = fmax(dmax, fmax(fabs(dx), fabs(dy)));
                        smax = fmax(smax, fmax(fabs(sv[s].x), fabs(sv[s].y)));
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
                        smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
                    }
                    if (dmax <= 1e-6 * smax) break;
                }
                conv = dmax <= 1e-4 * smax;
            }
            ok = conv;
            if (!conv) {
                // FP64 Cholesky of the same system in the slice's FP64 record
                double2* Kd = fb + (size_t)k * NPK;
                __syncwarp();
                for (int q = lane; q < NPK; q += 32) Kd[q] = to_d2(K[q]);
                __syncwarp();
                for (int p = lane; p < D; p += 32) Kd[tri(p, p)].x += lambda;
                ok = warp_chol<double2, double>(Kd, D, tol, lane);
                if (ok) {
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        const int p = lane + 32 * s;
                        sv[s] = p < D ? to_d2(K[NPK + p]) : make_double2(0.0, 0.0);
                    }
                    warp_chol_solve<double2, double, NS>(Kd, D, sv, lane);
                }
                if (lane == 0) atomicAdd(nref, 1ull);
            }
        } else {
            ok = warp_chol<V, T>(Lm, D, (T)tol, lane);
            if (ok) {
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    const int p = lane + 32 * s;
                    sv[s] = p < D ? to_d2(K[NPK + p]) : make_double2(0.0, 0.0);
                }
                warp_chol_solve<V, T, NS>(Lm, D, sv, lane);
            }
        }
        if (!ok && lane == 0) atomicAdd(nsing, 1ull);
        __syncwarp();
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const int p = lane + 32 * s;
            if (p < D) {
                if (ok) {
                    Zd[(size_t)k * D + p] = sv[s];
                    const V st = from_d2<V>(sv[s]);
                    Zt[(size_t)k * D + p] = st;
                    zt_s[p] = st;
                } else {
                    zt_s[p] = Zt[(size_t)k * D + p];
                }
            }
        }
        __syncwarp();
        // left environment update into the next order
        const int s0 = seg[k], s1 = seg[k + 1];
        for (int p = s0 + lane; p < s1; p += 32) {
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
