// Host-side drivers of the hot path, templated on compute type and rank.
// Each function only enqueues work on the context stream.
#pragma once

#include "bfc_gram_grp.cuh"
#include "bfc_gram_tc.cuh"
#include "bfc_internal.h"
#include "bfc_kernels.cuh"
#include "bfc_util.h"

namespace bfc {

inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T, int R> struct Path {
    typedef typename cvec<T>::type V;
    // the tensor-core Gram exists for the complex64 form with R * R <= 64
    static constexpr bool TC = sizeof(T) == 4 && R <= 8;
    // the grouped Gram's 4 x 4 tiles need R in {4, 8}
    static constexpr bool GRP = R == 4 || R == 8;

    static cudaError_t set_grp_attr()
    {
        if constexpr (GRP) {
            cudaError_t e = cudaFuncSetAttribute(k_mid_gram_grp<T, GRP ? R : 4, 0>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)GrpCfg<T, GRP ? R : 4>::SMEM);
            if (e != cudaSuccess) return e;
            return cudaFuncSetAttribute(k_mid_gram_grp<T, GRP ? R : 4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)GrpCfg<T, GRP ? R : 4>::SMEM);
        }
        return cudaSuccess;
    }

    // Whether middle level m runs the grouped Gram (fewer groups than the
    // context's ratio allows).
    static bool grouped(const Ctx* c, int m)
    {
        if constexpr (!GRP) return false;
        return level_grouped(c, m);
    }

    static cudaError_t set_tc_attr()
    {
        if constexpr (TC)
            return cudaFuncSetAttribute(k_mid_gram_tc<TC ? R : 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)TcGram::SMEM);
        return cudaSuccess;
    }

    static bfc_status configure(Ctx* c)
    {
        cudaError_t e = cudaFuncSetAttribute(k_mid_gram<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)GramCfg<T, R>::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_mid_solve<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SolveCfg<T, R>::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_mid_fallback<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SolveCfg<T, R>::SMEM);
        if (e == cudaSuccess && TC) e = set_tc_attr();
        if (e == cudaSuccess && GRP) e = set_grp_attr();
        if (e != cudaSuccess)
            return fail(c, BFC_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
        return BFC_OK;
    }

    // Bytes of the per-block normal-equation records (the larger of the
    // middle-slice and the outer-fiber layouts) and of the FP64 fallback area.
    static size_t record_bytes(int64_t n, int64_t S)
    {
        const size_t mid = (size_t)S * (GramCfg<T, R>::NPK + R * R) * sizeof(V);
        const size_t outer = (size_t)n * (R * (R + 1) / 2 + R) * sizeof(double2);
        return mid > outer ? mid : outer;
    }
    static size_t fallback_bytes(int64_t S)
    {
        return SolveCfg<T, R>::MIXED ? (size_t)S * SolveCfg<T, R>::NPK * sizeof(double2) : 0;
    }

    // One block-coordinate update of an outer factor (rows: S^1, cols: S^{L+2}).
    template <bool COLS>
    static bfc_status outer_level(Ctx* c, const V* A, int level, double2* zd, V* zt, V* Hn)
    {
        const int64_t n = c->n;
        double2* rec = (double2*)c->rec;
        {
            ProfScope ps(c, COLS ? "outer_cols_gram" : "outer_rows_gram");
            k_outer_gram<T, R><<<nblocks(n, 4), 128, 0, c->stream>>>(A, (const V*)c->tval[level], c->seg[level],
                                                                      (int)n, rec);
        }
        {
            ProfScope ps(c, COLS ? "outer_cols_solve" : "outer_rows_solve");
            k_outer_solve<T, R><<<nblocks(n, 64), 64, 0, c->stream>>>(rec, (int)n, c->P.lambda, c->ridge, zd, zt,
                                                                       c->d_count);
        }
        {
            ProfScope ps(c, COLS ? "outer_cols_post" : "outer_rows_post");
            k_outer_post<T, R, COLS><<<nblocks(n, 4), 128, 0, c->stream>>>(
                A, (const V*)c->tval[level], c->seg[level], (int)n, zt, COLS ? nullptr : c->nxt[0], Hn,
                COLS ? c->d_red : nullptr);
        }
        BFC_LAUNCH_CHECK(c, "outer level");
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
        const unsigned g = (unsigned)(S < (int64_t)c->num_sms * 16 ? S : (int64_t)c->num_sms * 16);
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
        const int64_t NR = c->N * R, S = c->S;
        const int L = c->L;
        V* W = (V*)c->W;
        V* H0 = (V*)c->H[0];
        V* H1 = (V*)c->H[1];
        BFC_TRY(right_envs(c));
        BFC_TRY(outer_level<false>(c, W, 0, c->z1d, (V*)c->z1t, H0));
        typedef GramCfg<T, R> GC;
        typedef SolveCfg<T, R> SC;
        const unsigned gsolve = (unsigned)((S + SC::WPB - 1) / SC::WPB);
        for (int m = 1; m <= L; ++m) {
            V* hin = (m - 1) & 1 ? H1 : H0;
            V* hout = m & 1 ? H1 : H0;
            {
                ProfScope ps(c, grouped(c, m) ? "mid_gram_grp" : "mid_gram");
                bool done = false;
                if constexpr (GRP) {
                    if (grouped(c, m)) {
                        const GroupLevel& gl = c->grp[m];
                        constexpr int RG = GRP ? R : 4;
                        typedef GsumCfg<T, RG> GS;
                        static_assert(GS::NTH == 128, "host block partition of the group sums");
                        // shared memory for the level's largest block (at most CAP entries)
                        const int cap = (int)std::min<int64_t>(gl.max_block, GS::CAP);
                        k_group_sums<T, RG><<<nblocks(gl.ngroups, GS::GB), GS::NTH,
                                              (size_t)cap * (RG + 1) * GS::VS, c->stream>>>(
                            hin, W + (size_t)m * NR, (const V*)c->tval[m], gl.gstart, (int)gl.ngroups, gl.by_col,
                            (V*)c->grec, cap);
                        if (gl.by_col)
                            k_mid_gram_grp<T, RG, 1><<<(unsigned)S, GrpCfg<T, RG>::NTH, GrpCfg<T, RG>::SMEM,
                                                       c->stream>>>((const V*)c->grec, gl.gseg, (V*)c->rec, (int)S);
                        else
                            k_mid_gram_grp<T, RG, 0><<<(unsigned)S, GrpCfg<T, RG>::NTH, GrpCfg<T, RG>::SMEM,
                                                       c->stream>>>((const V*)c->grec, gl.gseg, (V*)c->rec, (int)S);
                        ps.add_kernels(1);
                        done = true;
                    }
                }
                if constexpr (TC) {
                    if (!done && c->gram_tc) {
                        const unsigned g = (unsigned)(S < c->num_sms ? S : c->num_sms);
                        k_mid_gram_tc<TC ? R : 1><<<g, TcGram::NTH, TcGram::SMEM, c->stream>>>(
                            (const float2*)hin, (const float2*)(W + (size_t)m * NR), (const float2*)c->tval[m],
                            c->seg[m], (float2*)c->rec, (int)S, c->d_count + 5);
                        done = true;
                    }
                }
                if (!done)
                    k_mid_gram<T, R><<<(unsigned)S, GC::NTH, GC::SMEM, c->stream>>>(
                        hin, W + (size_t)m * NR, (const V*)c->tval[m], c->seg[m], (V*)c->rec, (int)S);
            }
            {
                ProfScope ps(c, "mid_solve");
                if (SC::MIXED) cudaMemsetAsync(c->d_count + 3, 0, sizeof(unsigned long long), c->stream);
                k_mid_solve<T, R><<<gsolve, 32 * SC::WPB, SC::SMEM, c->stream>>>(
                    (const V*)c->rec, hin, c->seg[m], c->nxt[m], hout, c->Zd + (size_t)(m - 1) * S * R * R,
                    (V*)c->Zt + (size_t)(m - 1) * S * R * R, c->fb, c->P.lambda, c->ridge, c->d_count,
                    c->d_count + 3, c->d_count + 2, c->fblist, (int)S, c->d_count + 5, c->inject == 1 ? 1 : 0);
            }
            if (SC::MIXED) {
                ProfScope ps(c, "mid_fallback");
                // a grid-stride loop over the listed slices (usually none): one
                // wave of blocks at most
                const unsigned gfb = std::min<unsigned>(gsolve, (unsigned)c->num_sms * SC::MINB);
                k_mid_fallback<T, R><<<gfb, 32 * SC::WPB, SC::SMEM, c->stream>>>(
                    (const V*)c->rec, hin, c->seg[m], c->nxt[m], hout, c->Zd + (size_t)(m - 1) * S * R * R,
                    (V*)c->Zt + (size_t)(m - 1) * S * R * R, c->fb, c->P.lambda, c->ridge, c->d_count,
                    c->d_count + 3, c->fblist, c->d_count + 1);   // + the fallbacks of the sweep
            }
        }
        BFC_LAUNCH_CHECK(c, "middle levels");
        V* hc = L & 1 ? H1 : H0;
        BFC_TRY(outer_level<true>(c, hc, L + 1, c->zLd, (V*)c->zLt, nullptr));
        {
            ProfScope ps(c, "reduce");
            launch_reduce_pairs(c->d_red, c->n, c->d_scalars + 0, c->stream);
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
        const unsigned g = (unsigned)(S < (int64_t)c->num_sms * 16 ? S : (int64_t)c->num_sms * 16);
        for (int m = 1; m <= L; ++m) {
            const int in = (m - 1) & 1, out = m & 1;
            ProfScope ps(c, "grad_mid");
            k_grad_mid<T, R><<<g, 128, 0, c->stream>>>(Hb[in], W + (size_t)m * NR, Rb[in], c->seg[m], c->nxt[m],
                                                        (const V*)c->Zt + (size_t)(m - 1) * S * R * R, Hb[out],
                                                        Rb[out], GZ + (size_t)(m - 1) * S * R * R, (int)S,
                                                        c->d_count + 5, c->inject == 1 ? 1 : 0);
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
