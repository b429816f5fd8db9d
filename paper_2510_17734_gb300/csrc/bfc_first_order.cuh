// First-order butterfly completion (ADAM, Alg. 3/4; ADF, Alg. 5 with the
// App. A.3 orthogonalization sweeps) and the O(n log n) butterfly
// matrix-vector product (Eq. (butterfly-mat-vec)), templated on the compute
// type T (float: complex64 environments, double: FP64) and the rank R.
//
// The sweeps keep the ALS sweep's data layout: every training entry has a
// position in each level order l = 0..L+1, W[l] holds the right environments
// w_l in order l, the left environment h_l travels from order l-1 to order
// l through nxt, and so does the ADF residual.  Factor updates happen in
// FP64 on the master factors, followed by the compute-type copy.
#pragma once

#include "bfc_fo.h"
#include "bfc_internal.h"
#include "bfc_kernels.cuh"
#include "bfc_path.cuh"
#include "bfc_util.h"

namespace bfc {

// One Alg. 3 update of a complex parameter s (two reals) with gradient g and
// moments (Re, Im pairs) in FP64.
__device__ __forceinline__ double2 adam_step(double2 s, double2 g, double2* __restrict__ Mp,
                                             double2* __restrict__ Vp, const AdamHyper& h)
{
    double2 m = *Mp, v = *Vp;
    m.x = h.beta1 * m.x + (1.0 - h.beta1) * g.x;
    m.y = h.beta1 * m.y + (1.0 - h.beta1) * g.y;
    v.x = h.beta2 * v.x + (1.0 - h.beta2) * (g.x * g.x);
    v.y = h.beta2 * v.y + (1.0 - h.beta2) * (g.y * g.y);
    *Mp = m;
    *Vp = v;
    s.x -= h.alpha * (m.x * h.inv1) / (sqrt(v.x * h.inv2) + h.sigma);
    s.y -= h.alpha * (m.y * h.inv1) / (sqrt(v.y * h.inv2) + h.sigma);
    return s;
}

// The value lane c of a warp holds for a register array indexed by c.
template <typename A, int R> __device__ __forceinline__ A pick(const A (&arr)[R], int c)
{
    A out = arr[0];
#pragma unroll
    for (int q = 1; q < R; ++q)
        if (q == c) out = arr[q];
    return out;
}

// ------------------------------------------------------------------ ADAM

// Outer factor of Alg. 4 (rows: S^1 with design w_0; columns: S^{L+2} with
// design h_{L+1}), one warp per fiber: gradient sum (x - t) conj(a) +
// lambda s at the current fiber, the Alg. 3 update, then (rows) h_1 = the new
// fiber into order 1 or (columns) the training residual partials with the
// new fiber.
template <typename T, int R, bool COLS>
__global__ void __launch_bounds__(256)
k_adam_outer(const typename cvec<T>::type* __restrict__ A, const typename cvec<T>::type* __restrict__ tv,
             const int32_t* __restrict__ seg, int nfib, double2* __restrict__ zd,
             typename cvec<T>::type* __restrict__ zt, double2* __restrict__ Mo, double2* __restrict__ Vo,
             AdamHyper hp, double lam, const int32_t* __restrict__ nxt, typename cvec<T>::type* __restrict__ Hn,
             double* __restrict__ part)
{
    typedef typename cvec<T>::type V;
    const int lane = threadIdx.x & 31;
    const int f = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (f >= nfib) return;
    const int s0 = seg[f], s1 = seg[f + 1];
    V s[R];
#pragma unroll
    for (int c = 0; c < R; ++c) s[c] = zt[(size_t)f * R + c];
    GradAcc<T> g[R];
#pragma unroll
    for (int c = 0; c < R; ++c) g[c].zero();
    for (int p = s0 + lane; p < s1; p += 32) {
        V a[R];
        load_row_v<V, R>(A, (size_t)p, a);
        V x = czero<V>();
#pragma unroll
        for (int c = 0; c < R; ++c) cmac(x, s[c], a[c]);
        const V t = tv[p];
        V rr;
        rr.x = x.x - t.x;
        rr.y = x.y - t.y;
#pragma unroll
        for (int c = 0; c < R; ++c) g[c].add_r_conj(rr, a[c]);
    }
#pragma unroll
    for (int c = 0; c < R; ++c) g[c].warp_sum();
    if (lane < R) {
        const GradAcc<T> gc = pick<GradAcc<T>, R>(g, lane);
        const size_t q = (size_t)f * R + lane;
        const double2 sd = zd[q];
        const double2 gd = make_double2((double)gc.x + lam * sd.x, (double)gc.y + lam * sd.y);
        const double2 ns = adam_step(sd, gd, Mo + q, Vo + q, hp);
        zd[q] = ns;
        zt[q] = from_d2<V>(ns);
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < R; ++c) s[c] = zt[(size_t)f * R + c];
    if constexpr (!COLS) {
        for (int p = s0 + lane; p < s1; p += 32) {
            const size_t o = (size_t)nxt[p];
#pragma unroll
            for (int c = 0; c < R; ++c) Hn[o * R + c] = s[c];
        }
    } else {
        double fit = 0.0, den = 0.0;
        for (int p = s0 + lane; p < s1; p += 32) {
            V a[R];
            load_row_v<V, R>(A, (size_t)p, a);
            V x = czero<V>();
#pragma unroll
            for (int c = 0; c < R; ++c) cmac(x, s[c], a[c]);
            const V t = tv[p];
            const double dx = (double)x.x - (double)t.x, dy = (double)x.y - (double)t.y;
            fit += dx * dx + dy * dy;
            den += (double)t.x * (double)t.x + (double)t.y * (double)t.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fit += __shfl_xor_sync(0xffffffffu, fit, o);
            den += __shfl_xor_sync(0xffffffffu, den, o);
        }
        if (lane == 0) {
            part[2 * f] = fit;
            part[2 * f + 1] = den;
        }
    }
}

// Middle factor of Alg. 4, one CTA per slice (grid-stride): the residual of
// every entry with the current slice, the gradient sum (x - t) conj(h (x) w)
// + lambda Z (threads own components, chunks of entries staged in shared
// memory), the Alg. 3 update of the slice, then h_{m+1} = h_m^T Z(new) into
// order m+1.
template <typename T, int R>
__global__ void __launch_bounds__(128)
k_adam_mid(const typename cvec<T>::type* __restrict__ H, const typename cvec<T>::type* __restrict__ Wm,
           const typename cvec<T>::type* __restrict__ tv, const int32_t* __restrict__ seg,
           const int32_t* __restrict__ nxt, double2* __restrict__ Zd, typename cvec<T>::type* __restrict__ Zt,
           double2* __restrict__ Mo, double2* __restrict__ Vo, AdamHyper hp, double lam,
           typename cvec<T>::type* __restrict__ Hn, int S)
{
    typedef typename cvec<T>::type V;
    constexpr int D = R * R;
    constexpr int CH = 128;
    constexpr int NQ = (D + 127) / 128;
    __shared__ V z_s[D];
    __shared__ V h_s[CH * R];
    __shared__ V w_s[CH * R];
    __shared__ V r_s[CH];
    const int tid = threadIdx.x;
    for (int k = blockIdx.x; k < S; k += gridDim.x) {
        const int s0 = seg[k], s1 = seg[k + 1];
        __syncthreads();
        for (int q = tid; q < D; q += blockDim.x) z_s[q] = Zt[(size_t)k * D + q];
        double2 g[NQ];
#pragma unroll
        for (int u = 0; u < NQ; ++u) g[u] = make_double2(0.0, 0.0);
        for (int base = s0; base < s1; base += CH) {
            const int cnt = min(CH, s1 - base);
            __syncthreads();
            if (tid < cnt) {
                const size_t p = (size_t)(base + tid);
                V h[R], w[R];
                load_row_v<V, R>(H, p, h);
                load_row_v<V, R>(Wm, p, w);
                V x = czero<V>();
#pragma unroll
                for (int a = 0; a < R; ++a) {
                    V hz = czero<V>();
#pragma unroll
                    for (int c = 0; c < R; ++c) cmac(hz, z_s[a * R + c], w[c]);
                    cmac(x, h[a], hz);
                }
                const V t = tv[p];
                V rr;
                rr.x = x.x - t.x;
                rr.y = x.y - t.y;
                r_s[tid] = rr;
#pragma unroll
                for (int c = 0; c < R; ++c) {
                    h_s[tid * R + c] = h[c];
                    w_s[tid * R + c] = w[c];
                }
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < NQ; ++u) {
                const int q = tid + 128 * u;
                if (q < D) {
                    const int pa = q / R, pc = q - pa * R;
                    V acc = czero<V>();
                    for (int e = 0; e < cnt; ++e) cmacc(acc, cmul(h_s[e * R + pa], w_s[e * R + pc]), r_s[e]);
                    g[u].x += (double)acc.x;
                    g[u].y += (double)acc.y;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < NQ; ++u) {
            const int q = tid + 128 * u;
            if (q < D) {
                const size_t o = (size_t)k * D + q;
                const double2 sd = Zd[o];
                const double2 gd = make_double2(g[u].x + lam * sd.x, g[u].y + lam * sd.y);
                const double2 ns = adam_step(sd, gd, Mo + o, Vo + o, hp);
                Zd[o] = ns;
                const V st = from_d2<V>(ns);
                Zt[o] = st;
                z_s[q] = st;
            }
        }
        __syncthreads();
        for (int p = s0 + tid; p < s1; p += blockDim.x) {
            V h[R];
            load_row_v<V, R>(H, (size_t)p, h);
            const size_t o = (size_t)nxt[p];
#pragma unroll
            for (int c = 0; c < R; ++c) {
                V acc = czero<V>();
#pragma unroll
                for (int a = 0; a < R; ++a) cmac(acc, h[a], z_s[a * R + c]);
                Hn[o * R + c] = acc;
            }
        }
    }
}

// ------------------------------------------------------------------- ADF

// Outer factor of Alg. 5, one warp per fiber: the residual G (rows: t - x
// from the current fiber; columns: carried in order L+1), the direction
// N = sum G conj(a) - lambda s, the exact step
// alpha = ||N||^2 / (sum |a . N|^2 + lambda ||N||^2), s += alpha N, and the
// new residual G - alpha a . N: into order 1 (rows) or as training residual
// partials (columns).
template <typename T, int R, bool COLS>
__global__ void __launch_bounds__(256)
k_adf_outer(const typename cvec<T>::type* __restrict__ A, const typename cvec<T>::type* __restrict__ tv,
            const typename cvec<T>::type* __restrict__ Gin, const int32_t* __restrict__ seg, int nfib,
            double2* __restrict__ zd, typename cvec<T>::type* __restrict__ zt, double lam,
            const int32_t* __restrict__ nxt, typename cvec<T>::type* __restrict__ Gn, double* __restrict__ part)
{
    typedef typename cvec<T>::type V;
    const int lane = threadIdx.x & 31;
    const int f = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (f >= nfib) return;
    const int s0 = seg[f], s1 = seg[f + 1];
    V s[R];
    double2 sd[R];
#pragma unroll
    for (int c = 0; c < R; ++c) {
        s[c] = zt[(size_t)f * R + c];
        sd[c] = zd[(size_t)f * R + c];
    }
    auto residual = [&](int p, const V (&a)[R]) {
        if constexpr (COLS) {
            return Gin[p];
        } else {
            V x = czero<V>();
#pragma unroll
            for (int c = 0; c < R; ++c) cmac(x, s[c], a[c]);
            const V t = tv[p];
            V g;
            g.x = t.x - x.x;
            g.y = t.y - x.y;
            return g;
        }
    };
    GradAcc<T> nacc[R];
#pragma unroll
    for (int c = 0; c < R; ++c) nacc[c].zero();
    for (int p = s0 + lane; p < s1; p += 32) {
        V a[R];
        load_row_v<V, R>(A, (size_t)p, a);
        const V gr = residual(p, a);
#pragma unroll
        for (int c = 0; c < R; ++c) nacc[c].add_r_conj(gr, a[c]);
    }
    double2 N[R];
    double nn = 0.0;
#pragma unroll
    for (int c = 0; c < R; ++c) {
        nacc[c].warp_sum();
        N[c] = make_double2((double)nacc[c].x - lam * sd[c].x, (double)nacc[c].y - lam * sd[c].y);
        nn += N[c].x * N[c].x + N[c].y * N[c].y;
    }
    double zz = 0.0;
    for (int p = s0 + lane; p < s1; p += 32) {
        V a[R];
        load_row_v<V, R>(A, (size_t)p, a);
        double zx = 0.0, zy = 0.0;
#pragma unroll
        for (int c = 0; c < R; ++c) {
            zx += (double)a[c].x * N[c].x - (double)a[c].y * N[c].y;
            zy += (double)a[c].x * N[c].y + (double)a[c].y * N[c].x;
        }
        zz += zx * zx + zy * zy;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zz += __shfl_xor_sync(0xffffffffu, zz, o);
    const double den = zz + lam * nn;
    const double alpha = den > 0.0 ? nn / den : 0.0;
    if (lane < R) {
        const double2 nc = pick<double2, R>(N, lane);
        const double2 sc = pick<double2, R>(sd, lane);
        const double2 ns = make_double2(sc.x + alpha * nc.x, sc.y + alpha * nc.y);
        zd[(size_t)f * R + lane] = ns;
        zt[(size_t)f * R + lane] = from_d2<V>(ns);
    }
    double fit = 0.0, dent = 0.0;
    for (int p = s0 + lane; p < s1; p += 32) {
        V a[R];
        load_row_v<V, R>(A, (size_t)p, a);
        const V gr = residual(p, a);
        double zx = 0.0, zy = 0.0;
#pragma unroll
        for (int c = 0; c < R; ++c) {
            zx += (double)a[c].x * N[c].x - (double)a[c].y * N[c].y;
            zy += (double)a[c].x * N[c].y + (double)a[c].y * N[c].x;
        }
        const double gx = (double)gr.x - alpha * zx, gy = (double)gr.y - alpha * zy;
        if constexpr (COLS) {
            const V t = tv[p];
            fit += gx * gx + gy * gy;
            dent += (double)t.x * (double)t.x + (double)t.y * (double)t.y;
        } else {
            Gn[nxt[p]] = from_d2<V>(make_double2(gx, gy));
        }
    }
    if constexpr (COLS) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fit += __shfl_xor_sync(0xffffffffu, fit, o);
            dent += __shfl_xor_sync(0xffffffffu, dent, o);
        }
        if (lane == 0) {
            part[2 * f] = fit;
            part[2 * f + 1] = dent;
        }
    }
}

// Middle factor of Alg. 5, one CTA per slice (grid-stride): the direction
// N = sum G conj(h (x) w) - lambda Z (threads own components), the exact
// step alpha = ||N||^2 / (sum |h^T N w|^2 + lambda ||N||^2), Z += alpha N,
// and the new residual G - alpha h^T N w into order m+1.
template <typename T, int R>
__global__ void __launch_bounds__(128)
k_adf_mid(const typename cvec<T>::type* __restrict__ H, const typename cvec<T>::type* __restrict__ Wm,
          const typename cvec<T>::type* __restrict__ Gin, const int32_t* __restrict__ seg,
          const int32_t* __restrict__ nxt, double2* __restrict__ Zd, typename cvec<T>::type* __restrict__ Zt,
          double lam, typename cvec<T>::type* __restrict__ Gn, int S)
{
    typedef typename cvec<T>::type V;
    constexpr int D = R * R;
    constexpr int CH = 128;
    constexpr int NQ = (D + 127) / 128;
    __shared__ V h_s[CH * R];
    __shared__ V w_s[CH * R];
    __shared__ V g_s[CH];
    __shared__ double2 n_s[D];
    __shared__ V nt_s[D];   // the direction in the compute type, for the per-entry products
    __shared__ double red[4];
    __shared__ double alpha_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    auto block_sum = [&](double v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();
        if (lane == 0) red[wid] = v;
        __syncthreads();
        return red[0] + red[1] + red[2] + red[3];
    };
    // z_e = h^T N w in the compute type (the entry's own precision)
    auto zval = [&](const V (&h)[R], const V (&w)[R]) {
        V z = czero<V>();
#pragma unroll
        for (int a = 0; a < R; ++a) {
            V nw = czero<V>();   // (N w)_a
#pragma unroll
            for (int c = 0; c < R; ++c) cmac(nw, nt_s[a * R + c], w[c]);
            cmac(z, h[a], nw);
        }
        return to_d2(z);
    };
    for (int k = blockIdx.x; k < S; k += gridDim.x) {
        const int s0 = seg[k], s1 = seg[k + 1];
        __syncthreads();   // the previous slice's readers of n_s are done
        double2 nq[NQ];
#pragma unroll
        for (int u = 0; u < NQ; ++u) nq[u] = make_double2(0.0, 0.0);
        for (int base = s0; base < s1; base += CH) {
            const int cnt = min(CH, s1 - base);
            __syncthreads();
            for (int x = tid; x < cnt * R; x += blockDim.x) {
                h_s[x] = H[(size_t)base * R + x];
                w_s[x] = Wm[(size_t)base * R + x];
            }
            for (int x = tid; x < cnt; x += blockDim.x) g_s[x] = Gin[base + x];
            __syncthreads();
#pragma unroll
            for (int u = 0; u < NQ; ++u) {
                const int q = tid + 128 * u;
                if (q < D) {
                    const int pa = q / R, pc = q - pa * R;
                    V acc = czero<V>();
                    for (int e = 0; e < cnt; ++e) cmacc(acc, cmul(h_s[e * R + pa], w_s[e * R + pc]), g_s[e]);
                    nq[u].x += (double)acc.x;
                    nq[u].y += (double)acc.y;
                }
            }
        }
        double nn = 0.0;
#pragma unroll
        for (int u = 0; u < NQ; ++u) {
            const int q = tid + 128 * u;
            if (q < D) {
                const double2 sd = Zd[(size_t)k * D + q];
                const double2 nv = make_double2(nq[u].x - lam * sd.x, nq[u].y - lam * sd.y);
                n_s[q] = nv;
                nt_s[q] = from_d2<V>(nv);
                nn += nv.x * nv.x + nv.y * nv.y;
            }
        }
        nn = block_sum(nn);   // its first barrier also publishes n_s
        double zz = 0.0;
        for (int p = s0 + tid; p < s1; p += blockDim.x) {
            V h[R], w[R];
            load_row_v<V, R>(H, (size_t)p, h);
            load_row_v<V, R>(Wm, (size_t)p, w);
            const double2 z = zval(h, w);
            zz += z.x * z.x + z.y * z.y;
        }
        zz = block_sum(zz);
        if (tid == 0) {
            const double den = zz + lam * nn;
            alpha_s = den > 0.0 ? nn / den : 0.0;
        }
        __syncthreads();
        const double alpha = alpha_s;
#pragma unroll
        for (int u = 0; u < NQ; ++u) {
            const int q = tid + 128 * u;
            if (q < D) {
                const size_t o = (size_t)k * D + q;
                const double2 sd = Zd[o], nv = n_s[q];
                const double2 ns = make_double2(sd.x + alpha * nv.x, sd.y + alpha * nv.y);
                Zd[o] = ns;
                Zt[o] = from_d2<V>(ns);
            }
        }
        for (int p = s0 + tid; p < s1; p += blockDim.x) {
            V h[R], w[R];
            load_row_v<V, R>(H, (size_t)p, h);
            load_row_v<V, R>(Wm, (size_t)p, w);
            const double2 z = zval(h, w);
            const V g = Gin[p];
            Gn[nxt[p]] = from_d2<V>(make_double2((double)g.x - alpha * z.x, (double)g.y - alpha * z.y));
        }
    }
}

// h_{m+1}(e) = h_m(e)^T Z[m][k] for the entries of every slice k, into order
// m+1 (one CTA per slice, grid-stride).
template <typename T, int R>
__global__ void __launch_bounds__(128)
k_h_next(const typename cvec<T>::type* __restrict__ H, const int32_t* __restrict__ seg,
         const int32_t* __restrict__ nxt, const typename cvec<T>::type* __restrict__ Zt,
         typename cvec<T>::type* __restrict__ Hn, int S)
{
    typedef typename cvec<T>::type V;
    __shared__ V z_s[R * R];
    for (int k = blockIdx.x; k < S; k += gridDim.x) {
        const int s0 = seg[k], s1 = seg[k + 1];
        if (s0 == s1) continue;
        __syncthreads();
        for (int q = threadIdx.x; q < R * R; q += blockDim.x) z_s[q] = Zt[(size_t)k * R * R + q];
        __syncthreads();
        for (int p = s0 + threadIdx.x; p < s1; p += blockDim.x) {
            V h[R];
            load_row_v<V, R>(H, (size_t)p, h);
            const size_t o = (size_t)nxt[p];
#pragma unroll
            for (int c = 0; c < R; ++c) {
                V acc = czero<V>();
#pragma unroll
                for (int a = 0; a < R; ++a) cmac(acc, h[a], z_s[a * R + c]);
                Hn[o * R + c] = acc;
            }
        }
    }
}

// h_1(e) = z1(i) for the entries of every row fiber i, into order 1.
template <typename T, int R>
__global__ void __launch_bounds__(256)
k_h1_rows(const int32_t* __restrict__ seg, int nfib, const typename cvec<T>::type* __restrict__ zt,
          const int32_t* __restrict__ nxt, typename cvec<T>::type* __restrict__ Hn)
{
    typedef typename cvec<T>::type V;
    const int lane = threadIdx.x & 31;
    const int f = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (f >= nfib) return;
    V s[R];
#pragma unroll
    for (int c = 0; c < R; ++c) s[c] = zt[(size_t)f * R + c];
    for (int p = seg[f] + lane; p < seg[f + 1]; p += 32) {
        const size_t o = (size_t)nxt[p];
#pragma unroll
        for (int c = 0; c < R; ++c) Hn[o * R + c] = s[c];
    }
}

// ---------------------------------------------------------------- matvec

// Y_{L+1}[p][q] = sum over the leaf of zL(j)^T v_q(j), p = j / b (the
// contraction of S^{L+2} with the vectors over j_L); one thread per (p, q).
template <typename T, int R>
__global__ void k_mv_leaf(const typename cvec<T>::type* __restrict__ zL, const double2* __restrict__ Vin, int b,
                          int nvec, int npre, typename cvec<T>::type* __restrict__ Y)
{
    typedef typename cvec<T>::type V;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)npre * nvec) return;
    const int p = (int)(idx / nvec), q = (int)(idx - (int64_t)p * nvec);
    V acc[R];
#pragma unroll
    for (int c = 0; c < R; ++c) acc[c] = czero<V>();
    for (int l = 0; l < b; ++l) {
        const int64_t j = (int64_t)p * b + l;
        const V v = from_d2<V>(Vin[j * nvec + q]);
#pragma unroll
        for (int c = 0; c < R; ++c) cmac(acc[c], zL[j * R + c], v);
    }
#pragma unroll
    for (int c = 0; c < R; ++c) Y[idx * R + c] = acc[c];
}

// Level m of the contraction (m = L .. 1): Y_m[k] = Z[m][k] T_m[g(k)], where
// T_L[g] = Y_{L+1}[g] with g = the column bits of k, and for m < L
// T_m[g] = Y_{m+1}[2g] + Y_{m+1}[2g + 1] (the sum over j_m) with g = k
// without its bit m (i_{L-m}).  One thread per (k, q).
template <typename T, int R>
__global__ void k_mv_level(const typename cvec<T>::type* __restrict__ Zm, const typename cvec<T>::type* __restrict__ Yin,
                           typename cvec<T>::type* __restrict__ Yout, int m, int L, int nvec, int S)
{
    typedef typename cvec<T>::type V;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)S * nvec) return;
    const int k = (int)(idx / nvec), q = (int)(idx - (int64_t)k * nvec);
    V tv[R];
    if (m == L) {
        const int64_t g = k & ((1 << L) - 1);
#pragma unroll
        for (int c = 0; c < R; ++c) tv[c] = Yin[(g * nvec + q) * R + c];
    } else {
        const int64_t g = ((int64_t)(k >> (m + 1)) << m) | (k & ((1 << m) - 1));
#pragma unroll
        for (int c = 0; c < R; ++c) {
            const V a = Yin[((2 * g) * nvec + q) * R + c], bq = Yin[((2 * g + 1) * nvec + q) * R + c];
            tv[c].x = a.x + bq.x;
            tv[c].y = a.y + bq.y;
        }
    }
    const V* Z = Zm + (size_t)k * R * R;
#pragma unroll
    for (int a = 0; a < R; ++a) {
        V acc = czero<V>();
#pragma unroll
        for (int c = 0; c < R; ++c) cmac(acc, Z[a * R + c], tv[c]);
        Yout[idx * R + a] = acc;
    }
}

// u_q(i) = z1(i)^T T_0[p_i], T_0[p] = Y_1[2p] + Y_1[2p + 1] (the sum over j_0)
// for L >= 1, or Y_1[0] (the leaf contraction) for L = 0; one thread per (i, q).
template <typename T, int R>
__global__ void k_mv_root(const typename cvec<T>::type* __restrict__ z1, const typename cvec<T>::type* __restrict__ Y1,
                          int b, int L, int nvec, int64_t n, double2* __restrict__ U)
{
    typedef typename cvec<T>::type V;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * nvec) return;
    const int64_t i = idx / nvec;
    const int q = (int)(idx - i * nvec);
    const int64_t p = i / b;
    V acc = czero<V>();
#pragma unroll
    for (int a = 0; a < R; ++a) {
        V tv;
        if (L == 0) {
            tv = Y1[(int64_t)q * R + a];
        } else {
            const V x = Y1[((2 * p) * nvec + q) * R + a], y = Y1[((2 * p + 1) * nvec + q) * R + a];
            tv.x = x.x + y.x;
            tv.y = x.y + y.y;
        }
        cmac(acc, z1[i * R + a], tv);
    }
    U[idx] = to_d2(acc);
}

// --------------------------------------------------------------- drivers

template <typename T, int R> struct FirstOrder {
    typedef typename cvec<T>::type V;

    static unsigned grid_slices(int64_t S) { return (unsigned)(S < 152 * 16 ? S : 152 * 16); }

    // u = X(S) V (Eq. (butterfly-mat-vec)) for nvec vectors on the device:
    // Vd, Ud n x nvec complex128; Y0, Y1 scratch of 2^{L+1} nvec R values.
    static bfc_status matvec(Ctx* c, int nvec, const double2* Vd, double2* Ud, V* Y0, V* Y1)
    {
        const int L = c->L;
        const int64_t npre = (int64_t)1 << L;
        const int64_t S = c->S;
        {
            ProfScope ps(c, "mv_leaf");
            const int64_t cnt = npre * nvec;
            k_mv_leaf<T, R><<<nblocks(cnt, 256), 256, 0, c->stream>>>((const V*)c->zLt, Vd, c->b, nvec, (int)npre, Y0);
        }
        V* yin = Y0;
        V* yout = Y1;
        for (int m = L; m >= 1; --m) {
            ProfScope ps(c, "mv_level");
            const int64_t cnt = S * nvec;
            k_mv_level<T, R><<<nblocks(cnt, 256), 256, 0, c->stream>>>(
                (const V*)c->Zt + (size_t)(m - 1) * S * R * R, yin, yout, m, L, nvec, (int)S);
            V* tmp = yin;
            yin = yout;
            yout = tmp;
        }
        {
            ProfScope ps(c, "mv_root");
            const int64_t cnt = c->n * nvec;
            k_mv_root<T, R><<<nblocks(cnt, 256), 256, 0, c->stream>>>((const V*)c->z1t, yin, c->b, L, nvec, c->n, Ud);
        }
        BFC_LAUNCH_CHECK(c, "matvec");
        return BFC_OK;
    }

    // One outer iteration of Alg. 4 (right environments, then S^1, the middle
    // factors and S^{L+2} in order) plus the training residual partials.
    static bfc_status adam_iter(Ctx* c, const AdamHyper& hp, double2* M, double2* Vm)
    {
        const int64_t n = c->n, NR = c->N * R, S = c->S;
        const int L = c->L;
        const double lam = c->P.lambda;
        V* W = (V*)c->W;
        V* Hb[2] = {(V*)c->H[0], (V*)c->H[1]};
        BFC_TRY((Path<T, R>::right_envs(c)));
        const size_t offZ = (size_t)n * R, offL = offZ + (size_t)L * S * R * R;
        {
            ProfScope ps(c, "adam_rows");
            k_adam_outer<T, R, false><<<nblocks(n, 8), 256, 0, c->stream>>>(
                W, (const V*)c->tval[0], c->seg[0], (int)n, c->z1d, (V*)c->z1t, M, Vm, hp, lam, c->nxt[0], Hb[0],
                nullptr);
        }
        for (int m = 1; m <= L; ++m) {
            ProfScope ps(c, "adam_mid");
            const size_t o = offZ + (size_t)(m - 1) * S * R * R;
            k_adam_mid<T, R><<<grid_slices(S), 128, 0, c->stream>>>(
                Hb[(m - 1) & 1], W + (size_t)m * NR, (const V*)c->tval[m], c->seg[m], c->nxt[m],
                c->Zd + (size_t)(m - 1) * S * R * R, (V*)c->Zt + (size_t)(m - 1) * S * R * R, M + o, Vm + o, hp, lam,
                Hb[m & 1], (int)S);
        }
        {
            ProfScope ps(c, "adam_cols");
            k_adam_outer<T, R, true><<<nblocks(n, 8), 256, 0, c->stream>>>(
                Hb[L & 1], (const V*)c->tval[L + 1], c->seg[L + 1], (int)n, c->zLd, (V*)c->zLt, M + offL,
                Vm + offL, hp, lam, nullptr, nullptr, c->d_red);
        }
        BFC_LAUNCH_CHECK(c, "adam iteration");
        return BFC_OK;
    }

    // Compute-type copy of FP64 factor values [off, off + cnt).
    static void refresh(Ctx* c, size_t off, int64_t cnt)
    {
        if constexpr (sizeof(T) == 4) {
            ProfScope ps(c, "d2f");
            launch_d2f(c->z1d + off, (float2*)c->z1t + off, cnt, c->stream);
        }
    }

    // One iteration of Alg. 5: right-to-left orthogonalization (App. A.3),
    // right environments, then S^1, the middle factors and S^{L+2}, each with
    // the exact-step update and (but S^{L+2}) the QR of its bond groups with
    // R moved into the next factor; the training residual partials last.
    static bfc_status adf_iter(Ctx* c)
    {
        const int64_t n = c->n, NR = c->N * R, S = c->S;
        const int L = c->L;
        const double lam = c->P.lambda;
        const size_t offZ = (size_t)n * R, offL = offZ + (size_t)L * S * R * R, slz = (size_t)S * R * R;
        V* W = (V*)c->W;
        V* Hb[2] = {(V*)c->H[0], (V*)c->H[1]};
        V* Gb[2] = {(V*)c->Rres[0], (V*)c->Rres[1]};
        {
            ProfScope ps(c, "adf_orth", L + 1);
            cudaError_t e = launch_rl_orthogonalize(c->z1d, c->Zd, c->zLd, n, L, c->b, R, c->stream);
            if (e != cudaSuccess) return fail(c, BFC_ECUDA, std::string("orthogonalization: ") + cudaGetErrorString(e));
        }
        refresh(c, 0, c->Pn);
        BFC_TRY((Path<T, R>::right_envs(c)));
        {
            ProfScope ps(c, "adf_rows");
            k_adf_outer<T, R, false><<<nblocks(n, 8), 256, 0, c->stream>>>(
                W, (const V*)c->tval[0], nullptr, c->seg[0], (int)n, c->z1d, (V*)c->z1t, lam, c->nxt[0], Gb[0], nullptr);
        }
        {
            ProfScope ps(c, "adf_qr");
            cudaError_t e = launch_canon_level(c->z1d, c->Zd, c->zLd, n, L, c->b, R, 0, c->stream);
            if (e != cudaSuccess) return fail(c, BFC_ECUDA, std::string("QR: ") + cudaGetErrorString(e));
        }
        refresh(c, 0, (int64_t)n * R);
        refresh(c, L >= 1 ? offZ : offL, L >= 1 ? (int64_t)slz : (int64_t)n * R);
        if (L >= 1) {
            ProfScope ps(c, "adf_h");
            k_h1_rows<T, R><<<nblocks(n, 8), 256, 0, c->stream>>>(c->seg[0], (int)n, (const V*)c->z1t, c->nxt[0], Hb[0]);
        }
        for (int m = 1; m <= L; ++m) {
            V* hin = Hb[(m - 1) & 1];
            V* hout = Hb[m & 1];
            {
                ProfScope ps(c, "adf_mid");
                k_adf_mid<T, R><<<grid_slices(S), 128, 0, c->stream>>>(
                    hin, W + (size_t)m * NR, Gb[(m - 1) & 1], c->seg[m], c->nxt[m], c->Zd + (size_t)(m - 1) * slz,
                    (V*)c->Zt + (size_t)(m - 1) * slz, lam, Gb[m & 1], (int)S);
            }
            {
                ProfScope ps(c, "adf_qr");
                cudaError_t e = launch_canon_level(c->z1d, c->Zd, c->zLd, n, L, c->b, R, m, c->stream);
                if (e != cudaSuccess) return fail(c, BFC_ECUDA, std::string("QR: ") + cudaGetErrorString(e));
            }
            refresh(c, offZ + (size_t)(m - 1) * slz, (int64_t)slz);
            refresh(c, m < L ? offZ + (size_t)m * slz : offL, m < L ? (int64_t)slz : (int64_t)n * R);
            {
                ProfScope ps(c, "adf_h");
                k_h_next<T, R><<<grid_slices(S), 128, 0, c->stream>>>(
                    hin, c->seg[m], c->nxt[m], (const V*)c->Zt + (size_t)(m - 1) * slz, hout, (int)S);
            }
        }
        {
            ProfScope ps(c, "adf_cols");
            const V* hc = L == 0 ? nullptr : Hb[L & 1];
            if (L == 0) {
                // L = 0: the column design is z1(i) itself, in the column order
                k_h1_rows<T, R><<<nblocks(n, 8), 256, 0, c->stream>>>(c->seg[0], (int)n, (const V*)c->z1t,
                                                                      c->nxt[0], Hb[0]);
                hc = Hb[0];
            }
            k_adf_outer<T, R, true><<<nblocks(n, 8), 256, 0, c->stream>>>(
                hc, (const V*)c->tval[L + 1], Gb[L & 1], c->seg[L + 1], (int)n, c->zLd, (V*)c->zLt, lam, nullptr,
                nullptr, c->d_red);
        }
        BFC_LAUNCH_CHECK(c, "adf iteration");
        return BFC_OK;
    }
};

template <typename T, int R> struct FoEntry {
    static bfc_status matvec(Ctx* c, int nvec, const double2* Vd, double2* Ud, void* y0, void* y1)
    {
        return FirstOrder<T, R>::matvec(c, nvec, Vd, Ud, (typename cvec<T>::type*)y0, (typename cvec<T>::type*)y1);
    }
    static constexpr FoOps ops{&matvec, &FirstOrder<T, R>::adam_iter, &FirstOrder<T, R>::adf_iter};
};

}  // namespace bfc
