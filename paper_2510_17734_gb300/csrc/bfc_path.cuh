// Host-side drivers of the hot path, templated on compute type and rank.
// Each function only enqueues work on the context stream.
#pragma once

#include "bfc_internal.h"
#include "bfc_kernels.cuh"
#include "bfc_util.h"

namespace bfc {

inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T, int R> struct Path {
    typedef typename cvec<T>::type V;

    static bfc_status configure(Ctx* c)
    {
        typedef MidCfg<T, R> C;
        cudaError_t e = cudaFuncSetAttribute(k_mid<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM);
        if (e != cudaSuccess)
            return fail(c, BFC_ECUDA, std::string("cudaFuncSetAttribute(k_mid): ") + cudaGetErrorString(e));
        return BFC_OK;
    }

    // Right environments w_L .. w_0 from the current factors (compute copies).
    static bfc_status right_envs(Ctx* c)
    {
        const int64_t N = c->N, NR = c->N * R, S = c->S;
        V* W = (V*)c->W;
        {
            ProfScope ps(c, "env_init");
            k_env_init<T, R><<<nblocks(NR, 256), 256, 0, c->stream>>>(W + (size_t)c->L * NR, (const V*)c->zLt,
                                                                       c->jL, N);
        }
        BFC_LAUNCH_CHECK(c, "env_init");
        const unsigned g = (unsigned)(S < 152 * 16 ? S : 152 * 16);
        for (int m = c->L; m >= 1; --m) {
            ProfScope ps(c, "env_right");
            k_env_right<T, R><<<g, 128, 0, c->stream>>>(W + (size_t)m * NR, W + (size_t)(m - 1) * NR,
                                                         (const V*)c->Zt + (size_t)(m - 1) * S * R * R,
                                                         c->seg[m], c->prv[m], (int)S);
        }
        BFC_LAUNCH_CHECK(c, "env_right");
        return BFC_OK;
    }

    // One ALS sweep (Alg. 1) + training residual partials (per column fiber).
    static bfc_status sweep(Ctx* c)
    {
        typedef MidCfg<T, R> C;
        const int64_t NR = c->N * R, S = c->S, n = c->n;
        const int L = c->L;
        V* W = (V*)c->W;
        V* H0 = (V*)c->H[0];
        V* H1 = (V*)c->H[1];
        BFC_TRY(right_envs(c));
        {
            ProfScope ps(c, "outer_rows");
            k_outer<T, R, false><<<nblocks(n, 4), 128, 0, c->stream>>>(
                W, (const V*)c->tval[0], c->seg[0], (int)n, c->P.lambda, c->z1d, (V*)c->z1t, c->nxt[0], H0,
                nullptr, c->d_count);
        }
        BFC_LAUNCH_CHECK(c, "outer_rows");
        for (int m = 1; m <= L; ++m) {
            V* hin = (m - 1) & 1 ? H1 : H0;
            V* hout = m & 1 ? H1 : H0;
            ProfScope ps(c, "mid_gram_solve");
            k_mid<T, R><<<(unsigned)S, C::NTH, C::SMEM, c->stream>>>(
                hin, W + (size_t)m * NR, (const V*)c->tval[m], c->seg[m], c->nxt[m], hout,
                c->Zd + (size_t)(m - 1) * S * R * R, (V*)c->Zt + (size_t)(m - 1) * S * R * R, c->P.lambda,
                c->d_count, (int)S);
        }
        BFC_LAUNCH_CHECK(c, "mid_gram_solve");
        V* hc = L & 1 ? H1 : H0;
        {
            ProfScope ps(c, "outer_cols");
            k_outer<T, R, true><<<nblocks(n, 4), 128, 0, c->stream>>>(
                hc, (const V*)c->tval[L + 1], c->seg[L + 1], (int)n, c->P.lambda, c->zLd, (V*)c->zLt, nullptr,
                nullptr, c->d_red, c->d_count);
        }
        BFC_LAUNCH_CHECK(c, "outer_cols");
        {
            ProfScope ps(c, "reduce");
            launch_reduce_pairs(c->d_red, n, c->d_scalars + 0, c->stream);
        }
        BFC_LAUNCH_CHECK(c, "reduce");
        return BFC_OK;
    }

    // Gradient of f into G (device, packed complex128); partial fits into part.
    static bfc_status grad(Ctx* c, double2* G, double* part)
    {
        const int64_t NR = c->N * R, S = c->S, n = c->n;
        const int L = c->L;
        V* W = (V*)c->W;
        V* Hb[2] = {(V*)c->H[0], (V*)c->H[1]};
        V* Rb[2] = {(V*)c->Rres[0], (V*)c->Rres[1]};
        BFC_TRY(right_envs(c));
        double2* G1 = G;
        double2* GZ = G + (size_t)n * R;
        double2* GL = GZ + (size_t)L * S * R * R;
        {
            ProfScope ps(c, "grad_rows");
            k_grad_rows<T, R><<<nblocks(n, 8), 256, 0, c->stream>>>(W, (const V*)c->tval[0], c->seg[0], (int)n,
                                                                     (const V*)c->z1t, c->nxt[0], Hb[0], Rb[0],
                                                                     G1, part);
        }
        BFC_LAUNCH_CHECK(c, "grad_rows");
        const unsigned g = (unsigned)(S < 152 * 16 ? S : 152 * 16);
        for (int m = 1; m <= L; ++m) {
            const int in = (m - 1) & 1, out = m & 1;
            ProfScope ps(c, "grad_mid");
            k_grad_mid<T, R><<<g, 128, 0, c->stream>>>(Hb[in], W + (size_t)m * NR, Rb[in], c->seg[m], c->nxt[m],
                                                        (const V*)c->Zt + (size_t)(m - 1) * S * R * R, Hb[out],
                                                        Rb[out], GZ + (size_t)(m - 1) * S * R * R, (int)S);
        }
        BFC_LAUNCH_CHECK(c, "grad_mid");
        {
            ProfScope ps(c, "grad_cols");
            k_grad_cols<T, R><<<nblocks(n, 8), 256, 0, c->stream>>>(Hb[L & 1], Rb[L & 1], c->seg[L + 1], (int)n,
                                                                     GL);
        }
        BFC_LAUNCH_CHECK(c, "grad_cols");
        return BFC_OK;
    }

    // Entry evaluation of M pairs (device arrays); out and/or residual partials.
    static bfc_status eval(Ctx* c, const int32_t* di, const int32_t* dj, int64_t M, double2* out,
                           const double2* tref, double* part, int nblk)
    {
        ProfScope ps(c, "eval");
        k_eval<T, R><<<nblk, 256, 0, c->stream>>>(di, dj, M, (const V*)c->z1t, (const V*)c->Zt, (const V*)c->zLt,
                                                   c->L, c->b, c->S, out, tref, part);
        BFC_LAUNCH_CHECK(c, "eval");
        return BFC_OK;
    }
};

}  // namespace bfc

#define BFC_INSTANTIATE(T, R) template struct bfc::Path<T, R>;
