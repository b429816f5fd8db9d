// C ABI of libbfc (include/bfc.h): context life cycle, data movement, the
// sweep / gradient / completion drivers and per-kernel profiling.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "bfc_fo.h"
#include "bfc_internal.h"
#include "bfc_ops.h"
#include "bfc_util.h"

namespace bfc {

static thread_local std::string g_create_err;

bfc_status fail(Ctx* ctx, bfc_status st, const std::string& msg)
{
    if (ctx) ctx->err = msg;
    else g_create_err = msg;
    return st;
}

bfc_status dalloc(Ctx* c, void** p, size_t bytes, const char* what)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(c, e == cudaErrorMemoryAllocation ? BFC_ENOMEM : BFC_ECUDA,
                    std::string("cudaMalloc(") + what + ", " + std::to_string(bytes) + " bytes): " +
                        cudaGetErrorString(e));
    }
    c->allocs.push_back(*p);
    return BFC_OK;
}

static void dfree(Ctx* c, void* p)
{
    if (!p) return;
    auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
    if (it != c->allocs.end()) c->allocs.erase(it);
    cudaFree(p);
}

bfc_status ensure_tmp(Ctx* c, size_t bytes)
{
    if (bytes <= c->tmp_cap) return BFC_OK;
    if (c->d_tmp) {
        cudaStreamSynchronize(c->stream);
        dfree(c, c->d_tmp);
        c->d_tmp = nullptr;
        c->tmp_cap = 0;
    }
    BFC_TRY(dalloc(c, &c->d_tmp, bytes, "scratch"));
    c->tmp_cap = bytes;
    return BFC_OK;
}

ProfScope::ProfScope(Ctx* ctx, const char* name, int k) : c(ctx), kernels(k)
{
    c->n_launch += k;
    if (!c->prof) return;
    for (size_t q = 0; q < c->prof_rec.size(); ++q)
        if (c->prof_rec[q].name == name) { rec = (int)q; break; }
    if (rec < 0) {
        c->prof_rec.push_back(ProfRecord{name, 0, 0.0});
        rec = (int)c->prof_rec.size() - 1;
    }
    if (c->ev_pool.empty()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { rec = -1; return; }
        c->ev_pool.push_back(e);
    }
    a = c->ev_pool.back();
    c->ev_pool.pop_back();
    cudaEventRecord(a, c->stream);
}

ProfScope::~ProfScope()
{
    if (rec < 0 || !a) return;
    cudaEvent_t b;
    if (c->ev_pool.empty()) {
        if (cudaEventCreate(&b) != cudaSuccess) { c->ev_pool.push_back(a); return; }
    } else {
        b = c->ev_pool.back();
        c->ev_pool.pop_back();
    }
    cudaEventRecord(b, c->stream);
    c->prof_pending.push_back(ProfPending{rec, kernels, a, b});
}

void prof_collect(Ctx* c)
{
    if (c->prof_pending.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (auto& p : c->prof_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            c->prof_rec[p.rec].launches += p.kernels;
            c->prof_rec[p.rec].total_ms += ms;
        }
        c->ev_pool.push_back(p.a);
        c->ev_pool.push_back(p.b);
    }
    c->prof_pending.clear();
}

// ------------------------------------------------------------------ helpers

static bool valid_sizes(int64_t n, int L, int b, int r)
{
    if (L < 0 || L > 24 || b < 1 || r < 1 || r > MAX_RANK || n < 1) return false;
    if (n != (int64_t)b << L) return false;
    if (n > (int64_t)1 << 30) return false;
    return true;
}

static bfc_status sync(Ctx* c)
{
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, BFC_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
    prof_collect(c);
    return BFC_OK;
}

static cudaMemcpyKind in_kind(const Ctx* c) { return c->P.values_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
static cudaMemcpyKind out_kind(const Ctx* c) { return c->P.values_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

// Refresh the compute-type copies of the factors from the FP64 masters.
static bfc_status refresh_copies(Ctx* c)
{
    if (!c->fp32) return BFC_OK;
    launch_d2f(c->z1d, (float2*)c->z1t, c->n * c->r, c->stream);
    launch_d2f(c->Zd, (float2*)c->Zt, (int64_t)c->L * c->S * c->r * c->r, c->stream);
    launch_d2f(c->zLd, (float2*)c->zLt, c->n * c->r, c->stream);
    BFC_LAUNCH_CHECK(c, "d2f");
    return BFC_OK;
}

// Sum of squares of the FP64 master factors into d_scalars[slot].
static bfc_status factor_sumsq(Ctx* c, int slot)
{
    const int nb = (int)std::min<int64_t>(1216, (c->Pn + 255) / 256);
    {
        ProfScope ps(c, "sumsq");
        launch_sumsq(c->z1d, c->Pn, c->d_red, nb, c->stream);  // factors are contiguous (one allocation)
    }
    {
        ProfScope ps(c, "reduce");
        launch_reduce_single(c->d_red, nb, c->d_scalars + slot, c->stream);
    }
    BFC_LAUNCH_CHECK(c, "sumsq");
    return BFC_OK;
}

// ------------------------------------------------------------------ create

struct Inputs {
    int64_t nnz;
    const int32_t *i, *j;
    const double* t;
    int64_t ntest;
    const int32_t *it, *jt;
    const double* tt;
    cudaMemcpyKind kind;
};

static bfc_status build(Ctx* c, const Inputs& in)
{
    const int64_t N = c->N, n = c->n, S = c->S;
    const int L = c->L, r = c->r;
    int dev = 0;
    BFC_CK(c, cudaGetDevice(&dev));
    BFC_CK(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev));
    BFC_CK(c, cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
    c->stream = c->own_stream;
    BFC_CK(c, cudaEventCreate(&c->ev0));
    BFC_CK(c, cudaEventCreate(&c->ev1));

    BFC_TRY(dalloc(c, (void**)&c->d_i, N * 4, "i"));
    BFC_TRY(dalloc(c, (void**)&c->d_j, N * 4, "j"));
    BFC_TRY(dalloc(c, (void**)&c->d_t, N * 16, "t"));
    BFC_CK(c, cudaMemcpyAsync(c->d_i, in.i, N * 4, in.kind, c->stream));
    BFC_CK(c, cudaMemcpyAsync(c->d_j, in.j, N * 4, in.kind, c->stream));
    BFC_CK(c, cudaMemcpyAsync(c->d_t, in.t, N * 16, in.kind, c->stream));
    if (c->NT > 0) {
        BFC_TRY(dalloc(c, (void**)&c->d_it, c->NT * 4, "it"));
        BFC_TRY(dalloc(c, (void**)&c->d_jt, c->NT * 4, "jt"));
        BFC_TRY(dalloc(c, (void**)&c->d_tt, c->NT * 16, "tt"));
        BFC_CK(c, cudaMemcpyAsync(c->d_it, in.it, c->NT * 4, in.kind, c->stream));
        BFC_CK(c, cudaMemcpyAsync(c->d_jt, in.jt, c->NT * 4, in.kind, c->stream));
        BFC_CK(c, cudaMemcpyAsync(c->d_tt, in.tt, c->NT * 16, in.kind, c->stream));
    }
    BFC_TRY(dalloc(c, (void**)&c->d_scalars, 16 * sizeof(double), "scalars"));
    BFC_TRY(dalloc(c, (void**)&c->d_count, 8 * sizeof(unsigned long long), "counters"));
    BFC_CK(c, cudaMemsetAsync(c->d_count, 0, 8 * sizeof(unsigned long long), c->stream));
    c->red_cap = std::max<int64_t>(2 * n, 8192);
    BFC_TRY(dalloc(c, (void**)&c->d_red, c->red_cap * sizeof(double), "reduction"));

    // validation: index range, finite values
    int* dflag = (int*)c->d_count;
    BFC_CK(c, cudaMemsetAsync(dflag, 0, sizeof(int), c->stream));
    launch_check_entries(c->d_i, c->d_j, c->d_t, N, n, dflag, c->stream);
    launch_check_entries(c->d_it, c->d_jt, c->d_tt, c->NT, n, dflag, c->stream);
    BFC_LAUNCH_CHECK(c, "check_entries");
    int hflag = 0;
    BFC_CK(c, cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    BFC_TRY(sync(c));
    if (hflag & 1) return fail(c, BFC_EINVAL, "an index is outside [0, n)");
    if (hflag & 2) return fail(c, BFC_EINVAL, "a value is NaN or Inf");

    // level orders
    SortScratch ss;
    const int64_t T = (N + RS_TILE - 1) / RS_TILE;
    std::vector<void*> temps;
    auto tmp = [&](void** p, size_t bytes, const char* w) -> bfc_status {
        BFC_TRY(dalloc(c, p, bytes, w));
        temps.push_back(*p);
        return BFC_OK;
    };
    BFC_TRY(tmp((void**)&ss.k0, N * 4, "sort keys"));
    BFC_TRY(tmp((void**)&ss.k1, N * 4, "sort keys"));
    BFC_TRY(tmp((void**)&ss.v0, N * 4, "sort vals"));
    BFC_TRY(tmp((void**)&ss.v1, N * 4, "sort vals"));
    BFC_TRY(tmp((void**)&ss.counts, (size_t)256 * T * 4, "sort counts"));
    const int NL = L + 2;
    std::vector<int32_t*>& perm = c->perm;
    std::vector<int32_t*> pos(NL);
    perm.assign(NL, nullptr);
    c->seg.assign(NL, nullptr);
    c->tval.assign(NL, nullptr);
    c->nxt.assign(L + 1, nullptr);
    c->prv.assign(L + 1, nullptr);
    c->grp.assign(NL, GroupLevel{});
    std::vector<uint32_t> hkeys;
    for (int l = 0; l < NL; ++l) {
        const int64_t K = (l == 0 || l == L + 1) ? n : S;
        BFC_TRY(dalloc(c, (void**)&perm[l], N * 4, "perm"));
        BFC_TRY(tmp((void**)&pos[l], N * 4, "pos"));
        BFC_TRY(dalloc(c, (void**)&c->seg[l], (K + 1) * 4, "segments"));
        // + 16 bytes: the tensor-core Gram's bulk copies round their end up to
        // a 16-byte boundary
        BFC_TRY(dalloc(c, &c->tval[l], N * c->vsz + 16, "level values"));
        // middle levels: inside a slice, entries of one row (levels m with
        // 2m <= L+1, where a slice's block has fewer rows than columns) or of
        // one column are contiguous; they share h_m (resp. w_m)
        int64_t loc = 0;
        int by_col = 0;
        if (l >= 1 && l <= L) {
            by_col = 2 * l > L + 1;
            loc = by_col ? ((int64_t)c->b << (L - l)) : ((int64_t)c->b << (l - 1));
            if ((double)S * (double)loc >= 2147483647.0) loc = 0;
        }
        uint32_t* skeys = nullptr;
        BFC_CK(c, sort_level(c->d_i, c->d_j, N, l, L, c->b, K, loc, by_col, c->stream, ss, perm[l], c->seg[l],
                             &skeys));
        if (loc > 0) {
            // row / column groups of the level: entry offsets and the first
            // group of every slice
            hkeys.resize(N);
            BFC_CK(c, cudaMemcpyAsync(hkeys.data(), skeys, N * 4, cudaMemcpyDeviceToHost, c->stream));
            BFC_TRY(sync(c));
            std::vector<int32_t> gst, gsg(S + 1, 0);
            gst.reserve(N / 2 + 1);
            for (int64_t p = 0; p < N; ++p)
                if (p == 0 || hkeys[p] != hkeys[p - 1]) gst.push_back((int32_t)p);
            const int64_t G = (int64_t)gst.size();
            GroupLevel& gl = c->grp[l];
            gl.by_col = by_col;
            gl.ngroups = G;
            const double ratio = c->gram_tc ? c->grp_max_ratio : c->grp_cuda_ratio;
            if ((c->r == 4 || c->r == 8) && c->P.gram_impl == 0 && (double)G < ratio * (double)N) {
                gst.push_back((int32_t)N);
                // the largest entry range of a k_group_sums block (its shared-memory staging)
                const int64_t gpb = 128 / c->r;
                for (int64_t g0 = 0; g0 < G; g0 += gpb)
                    gl.max_block = std::max(gl.max_block, (int64_t)gst[std::min(g0 + gpb, G)] - gst[g0]);
                int64_t g = 0;
                for (int64_t k = 0; k <= S; ++k) {
                    while (g < G && (int64_t)(hkeys[gst[g]] / (uint64_t)loc) < k) ++g;
                    gsg[k] = (int32_t)g;
                }
                BFC_TRY(dalloc(c, (void**)&gl.gstart, (size_t)(G + 1) * 4, "group offsets"));
                BFC_TRY(dalloc(c, (void**)&gl.gseg, (size_t)(S + 1) * 4, "slice group offsets"));
                BFC_CK(c, cudaMemcpyAsync(gl.gstart, gst.data(), (size_t)(G + 1) * 4, cudaMemcpyHostToDevice,
                                          c->stream));
                BFC_CK(c, cudaMemcpyAsync(gl.gseg, gsg.data(), (size_t)(S + 1) * 4, cudaMemcpyHostToDevice,
                                          c->stream));
                BFC_TRY(sync(c));   // the host vectors go out of scope
            } else {
                // the level runs a per-entry Gram: its slices keep the entries
                // in input order (a row- or column-sorted slice makes the
                // per-entry partial sums coherent, and their rounding larger)
                BFC_CK(c, sort_level(c->d_i, c->d_j, N, l, L, c->b, K, 0, 0, c->stream, ss, perm[l], c->seg[l],
                                     nullptr));
            }
        }
        launch_invert(perm[l], N, pos[l], c->stream);
        launch_gather_values(c->d_t, perm[l], N, c->tval[l], c->fp32, c->stream);
        BFC_LAUNCH_CHECK(c, "prep");
    }
    // duplicates: columns within each row segment must be distinct
    int32_t* jrow = ss.v1;  // free after the sorts
    launch_gather_i32(c->d_j, perm[0], N, jrow, c->stream);
    BFC_CK(c, cudaMemsetAsync(dflag, 0, sizeof(int), c->stream));
    launch_row_dups(c->seg[0], jrow, n, dflag, c->stream);
    BFC_LAUNCH_CHECK(c, "row_dups");
    for (int l = 0; l <= L; ++l) {
        BFC_TRY(dalloc(c, (void**)&c->nxt[l], N * 4, "nxt"));
        launch_compose(perm[l], pos[l + 1], N, c->nxt[l], c->stream);
        if (l >= 1) {
            BFC_TRY(dalloc(c, (void**)&c->prv[l], N * 4, "prv"));
            launch_compose(perm[l], pos[l - 1], N, c->prv[l], c->stream);
        }
    }
    BFC_TRY(dalloc(c, (void**)&c->jL, N * 4, "jL"));
    launch_gather_i32(c->d_j, perm[L], N, c->jL, c->stream);
    BFC_LAUNCH_CHECK(c, "maps");
    BFC_CK(c, cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    BFC_TRY(sync(c));
    for (void* p : temps) dfree(c, p);
    if (hflag & 4) return fail(c, BFC_EINVAL, "duplicate (i, j) pair in the training set");

    // environments
    BFC_TRY(dalloc(c, &c->W, (size_t)(L + 1) * N * r * c->vsz + 16, "right environments"));
    for (int q = 0; q < 2; ++q) {
        BFC_TRY(dalloc(c, &c->H[q], (size_t)N * r * c->vsz + 16, "left environments"));
        BFC_TRY(dalloc(c, &c->Rres[q], (size_t)N * c->vsz, "residuals"));
    }
    // factors: one allocation, FP64 master [z1 | Z | zL]
    BFC_TRY(dalloc(c, (void**)&c->z1d, (size_t)c->Pn * 16, "factors"));
    c->Zd = c->z1d + n * r;
    c->zLd = c->Zd + (size_t)L * S * r * r;
    BFC_CK(c, cudaMemsetAsync(c->z1d, 0, (size_t)c->Pn * 16, c->stream));
    if (c->fp32) {
        void* ft;
        BFC_TRY(dalloc(c, &ft, (size_t)c->Pn * 8, "factors c64"));
        c->z1t = ft;
        c->Zt = (float2*)ft + n * r;
        c->zLt = (float2*)c->Zt + (size_t)L * S * r * r;
        BFC_CK(c, cudaMemsetAsync(ft, 0, (size_t)c->Pn * 8, c->stream));
    } else {
        c->z1t = c->z1d;
        c->Zt = c->Zd;
        c->zLt = c->zLd;
    }
    const Ops* ops = get_ops(c->fp32, r);
    BFC_TRY(dalloc(c, &c->rec, ops->record_bytes(n, S), "normal-equation records"));
    // group records [s | M | v] of the grouped Gram (ranks 4 and 8): sized for
    // the largest level whose order was grouped
    if ((r == 4 || r == 8) && c->P.gram_impl == 0) {
        int64_t gmax = 0;
        for (const GroupLevel& gl : c->grp)
            if (gl.gstart) gmax = std::max(gmax, gl.ngroups);
        // record [s | M (with 64 bytes between its two row halves) | v]
        const size_t rec_vals = (size_t)(2 * r + r * r) + 64 / c->vsz;
        if (gmax > 0) BFC_TRY(dalloc(c, &c->grec, (size_t)gmax * rec_vals * c->vsz, "group records"));
    }
    const size_t fbb = ops->fallback_bytes(S);
    if (fbb > 0 && L > 0) {
        BFC_TRY(dalloc(c, (void**)&c->fb, fbb, "FP64 fallback records"));
        BFC_TRY(dalloc(c, (void**)&c->fblist, (size_t)S * sizeof(int32_t), "fallback list"));
    }
    BFC_TRY(ops->configure(c));
    return sync(c);
}

static bfc_status create_impl(const bfc_params* params, const Inputs& in, bfc_ctx** out)
{
    if (out) *out = nullptr;
    if (!params || !out) return fail(nullptr, BFC_EINVAL, "null argument");
    const bfc_params& p = *params;
    if (!valid_sizes(p.n, p.L, p.b, p.r))
        return fail(nullptr, BFC_EINVAL, "invalid sizes: need n = b * 2^L, 0 <= L <= 24, 1 <= r <= 12");
    if (!(p.lambda >= 0.0) || !isfinite(p.lambda)) return fail(nullptr, BFC_EINVAL, "lambda must be finite and >= 0");
    if (!isfinite(p.ridge_rel)) return fail(nullptr, BFC_EINVAL, "ridge_rel must be finite");
    if (p.prec != BFC_PREC_FP64 && p.prec != BFC_PREC_C64_FP64SOLVE)
        return fail(nullptr, BFC_EINVAL, "unknown precision");
    if (p.gram_impl < 0 || p.gram_impl > 2) return fail(nullptr, BFC_EINVAL, "gram_impl must be 0, 1 or 2");
    if (!(p.group_ratio == p.group_ratio)) return fail(nullptr, BFC_EINVAL, "group_ratio is NaN");
    if (p.max_sweeps < 0 || p.refine_sweeps < 0 || p.lr_sweeps < 0 || p.lr_rank < 0)
        return fail(nullptr, BFC_EINVAL, "sweep counts and lr_rank must be >= 0");
    if (p.init_kind < 0 || p.init_kind > 2) return fail(nullptr, BFC_EINVAL, "init_kind must be 0, 1 or 2");
    if (p.lr2bf_oversample < 0) return fail(nullptr, BFC_EINVAL, "lr2bf_oversample must be >= 0");
    if (in.nnz <= 0 || in.nnz >= ((int64_t)1 << 31) - 1) return fail(nullptr, BFC_EINVAL, "nnz must be in [1, 2^31-2]");
    if (in.ntest < 0 || in.ntest >= ((int64_t)1 << 31) - 1) return fail(nullptr, BFC_EINVAL, "bad ntest");
    if (!in.i || !in.j || !in.t) return fail(nullptr, BFC_EINVAL, "null training data");
    if (in.ntest > 0 && (!in.it || !in.jt || !in.tt)) return fail(nullptr, BFC_EINVAL, "null test data");
    Ctx* c = new Ctx();
    c->P = p;
    c->n = p.n;
    c->L = p.L;
    c->b = p.b;
    c->r = p.r;
    c->S = (int64_t)1 << (p.L + 1);
    c->N = in.nnz;
    c->NT = in.ntest;
    c->Pn = bfc_num_params(p.n, p.L, p.b, p.r);
    c->fp32 = p.prec == BFC_PREC_C64_FP64SOLVE;
    c->vsz = c->fp32 ? 8 : 16;
    c->ridge = p.ridge_rel > 0.0 ? p.ridge_rel : (p.ridge_rel == 0.0 && c->fp32 ? 9.5367431640625e-07 : 0.0);
    c->gram_tc = c->fp32 && p.gram_impl != 1 && p.r <= 8;
    // grouped Gram (gram_impl 0) at the middle levels with few row / column
    // groups per entry: below this ratio against the tensor-core kernel (a
    // group's compensated Kronecker update and its sums cost about what seven
    // entries cost there: at n = 65536 a level of 0.07 groups per entry is
    // faster grouped, one of 0.14 on the tensor cores), below 0.9 against the
    // per-entry CUDA-core kernel
    c->grp_max_ratio = p.group_ratio > 0.0 ? p.group_ratio : (p.group_ratio < 0.0 ? 0.0 : 0.1);
    c->grp_cuda_ratio = p.group_ratio > 0.0 ? p.group_ratio : (p.group_ratio < 0.0 ? 0.0 : 0.9);
    bfc_status st = build(c, in);
    if (st != BFC_OK) {
        g_create_err = c->err;
        bfc_destroy((bfc_ctx*)c);
        return st;
    }
    *out = (bfc_ctx*)c;
    return BFC_OK;
}

// ---------------------------------------------------------------- sweeps

// Failure injection of the tests, kind 2: the device error word is raised
// from the host, as if a bounded device wait had expired.
static bfc_status inject_error_word(Ctx* c)
{
    if (c->inject != 2) return BFC_OK;
    static const unsigned long long one = 1ull;
    BFC_CK(c, cudaMemcpyAsync(c->d_count + 5, &one, sizeof(one), cudaMemcpyHostToDevice, c->stream));
    return BFC_OK;
}

static bfc_status collect_stats(Ctx* c, bfc_sweep_stats* out, float ms)
{
    double hs[8];
    unsigned long long hc[6];
    BFC_TRY(inject_error_word(c));
    BFC_CK(c, cudaMemcpyAsync(hs, c->d_scalars, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    BFC_CK(c, cudaMemcpyAsync(hc, c->d_count, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    BFC_TRY(sync(c));
    if (hc[5] != 0) {
        // a bounded wait inside the tensor-core Gram or on a bulk copy of the
        // solve expired: the sweep's results are undefined; clear the flag so
        // the context stays usable
        BFC_CK(c, cudaMemsetAsync(c->d_count + 5, 0, sizeof(unsigned long long), c->stream));
        BFC_TRY(sync(c));
        return fail(c, BFC_ETIMEOUT, "a bounded device wait expired (tensor-core Gram or bulk copy)");
    }
    if (out) {
        out->sweep = c->sweeps_done;
        out->train_rel_err = hs[1] > 0 ? sqrt(hs[0] / hs[1]) : sqrt(hs[0]);
        out->test_rel_err = c->NT > 0 ? (hs[4] > 0 ? sqrt(hs[3] / hs[4]) : sqrt(hs[3])) : -1.0;
        out->objective = 0.5 * hs[0] + 0.5 * c->P.lambda * hs[2];
        out->sweep_ms = ms;
        out->entries_per_s = ms > 0 ? (double)c->N / (ms * 1e-3) : 0.0;
        out->singular_slices = (int64_t)hc[0];
        out->refined_fallbacks = (int64_t)hc[1];
        out->refine_steps = (int64_t)hc[2];
        out->batch_launches = 0;
    }
    if (!isfinite(hs[0])) return fail(c, BFC_ENONFINITE, "training residual is not finite");
    return BFC_OK;
}

static bfc_status test_error(Ctx* c, int slot)
{
    if (c->NT <= 0) return BFC_OK;
    const Ops* ops = get_ops(c->fp32, c->r);
    const int nb = (int)std::min<int64_t>(1216, (c->NT + 255) / 256);
    BFC_TRY(ops->eval(c, c->d_it, c->d_jt, c->NT, nullptr, c->d_tt, c->d_red, nb));
    {
        ProfScope ps(c, "reduce");
        launch_reduce_pairs(c->d_red, nb, c->d_scalars + slot, c->stream);
    }
    BFC_LAUNCH_CHECK(c, "reduce");
    return BFC_OK;
}

// Device work of one sweep on c->stream: kernels and memsets only, so it can
// be captured into a graph.
static bfc_status sweep_enqueue(Ctx* c)
{
    const Ops* ops = get_ops(c->fp32, c->r);
    BFC_CK(c, cudaMemsetAsync(c->d_count, 0, 3 * sizeof(unsigned long long), c->stream));
    BFC_TRY(ops->sweep(c));
    BFC_TRY(factor_sumsq(c, 2));
    BFC_TRY(test_error(c, 3));
    return BFC_OK;
}

// Wait for an enqueued sweep and read its statistics.
static bfc_status sweep_finish(Ctx* c, bfc_sweep_stats* out, int64_t launched)
{
    c->sweeps_done += 1;
    BFC_TRY(sync(c));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    BFC_TRY(collect_stats(c, out, ms));
    if (out) {
        out->launches = launched;
        out->gram_impl = c->fp32 ? (c->gram_tc ? 0 : 1) : -1;
    }
    return BFC_OK;
}

static bfc_status capture_sweep(Ctx* c);

// One sweep and its statistics.  With `replay`, a context that is not
// profiling launches its captured sweep graph (captured on first use; the
// kernels and their order are those of the direct path), which removes the
// per-kernel launch cost of the 12 + 5 L kernels.
static bfc_status sweep_impl(Ctx* c, bfc_sweep_stats* out, bool replay = false)
{
    const int64_t launched0 = c->n_launch;
    if (replay && !c->prof) BFC_TRY(capture_sweep(c));
    const bool graph = replay && !c->prof && c->sweep_graph && c->graph_tc == c->gram_tc;
    BFC_CK(c, cudaEventRecord(c->ev0, c->stream));
    if (graph) {
        BFC_CK(c, cudaGraphLaunch(c->sweep_graph, c->stream));
        c->n_launch += c->graph_launches;
    } else {
        BFC_TRY(sweep_enqueue(c));
    }
    BFC_CK(c, cudaEventRecord(c->ev1, c->stream));
    return sweep_finish(c, out, c->n_launch - launched0);
}

static void drop_graph(Ctx* c)
{
    if (c->sweep_graph) cudaGraphExecDestroy(c->sweep_graph);
    if (c->sweep_graph_src) cudaGraphDestroy(c->sweep_graph_src);
    c->sweep_graph = nullptr;
    c->sweep_graph_src = nullptr;
}

// Capture one sweep of this context into a graph (once per Gram kernel
// choice).  Leaves no graph and returns BFC_OK when the stream cannot be
// captured (the legacy default stream); the caller then enqueues directly.
static bfc_status capture_sweep(Ctx* c)
{
    if (c->sweep_graph && c->graph_tc == c->gram_tc) return BFC_OK;
    drop_graph(c);
    if (c->prof) return BFC_OK;   // profiling records events per kernel: no graph
    const int64_t l0 = c->n_launch;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return BFC_OK;
    }
    const bfc_status st = sweep_enqueue(c);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (st != BFC_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(c, BFC_ECUDA, std::string("sweep capture: ") + cudaGetErrorString(e));
    const cudaError_t e2 = cudaGraphInstantiate(&c->sweep_graph, g, 0);
    if (e2 != cudaSuccess) {
        cudaGraphDestroy(g);
        c->sweep_graph = nullptr;
        return fail(c, BFC_ECUDA, std::string("sweep graph: ") + cudaGetErrorString(e2));
    }
    c->sweep_graph_src = g;   // kept: the batch embeds it in one graph per round
    c->graph_launches = c->n_launch - l0;   // kernels recorded by the capture
    c->n_launch = l0;                        // nothing ran yet
    c->graph_tc = c->gram_tc;
    return BFC_OK;
}

// Gradient of f (with lambda S when include_reg) into the device vector G;
// hs[0] = sum |x - t|^2 over the training entries, hs[2] = ||S||^2.
static bfc_status grad_into(Ctx* c, int include_reg, double2* G, double* hs)
{
    double* part = c->d_red;  // per-fiber partial fits
    const Ops* ops = get_ops(c->fp32, c->r);
    BFC_TRY(ops->grad(c, G, part));
    {
        ProfScope ps(c, "reduce");
        launch_reduce_single(part, c->n, c->d_scalars + 0, c->stream);
    }
    BFC_TRY(factor_sumsq(c, 2));
    if (include_reg) launch_axpy((double*)G, (const double*)c->z1d, c->P.lambda, 2 * c->Pn, c->stream);
    BFC_LAUNCH_CHECK(c, "grad tail");
    BFC_TRY(inject_error_word(c));
    unsigned long long terr = 0;
    BFC_CK(c, cudaMemcpyAsync(hs, c->d_scalars, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    BFC_CK(c, cudaMemcpyAsync(&terr, c->d_count + 5, sizeof(terr), cudaMemcpyDeviceToHost, c->stream));
    BFC_TRY(sync(c));
    if (terr != 0) {
        // a bounded wait on a bulk copy of the gradient sweep expired: the
        // gradient is undefined; clear the flag so the context stays usable
        BFC_CK(c, cudaMemsetAsync(c->d_count + 5, 0, sizeof(unsigned long long), c->stream));
        BFC_TRY(sync(c));
        return fail(c, BFC_ETIMEOUT, "gradient sweep: a bounded device wait expired");
    }
    return BFC_OK;
}

// Dot product of two device vectors of n doubles, returned on the host.
static bfc_status ddot(Ctx* c, const double* a, const double* b, int64_t n, double* out)
{
    const int nb = (int)std::min<int64_t>(1216, (n + 255) / 256);
    launch_dot(a, b, n, c->d_red, nb, c->d_scalars + 8, c->stream);
    BFC_LAUNCH_CHECK(c, "dot");
    BFC_CK(c, cudaMemcpyAsync(out, c->d_scalars + 8, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return sync(c);
}

// Limited-memory BFGS on the 2P real parameters (the packed factors viewed as
// doubles) of the regularized objective f (Eq. BF_objective + lambda/2 ||S||^2),
// with gradients from the gradient sweep (Eqs. grad_butterfly_*).  Two-loop
// recursion (Nocedal and Wright, Alg. 7.4) with memory m and H0 = gamma I,
// gamma = s^T y / y^T y of the newest pair; backtracking Armijo line search
// (c1 = 1e-4, halving, at most 30 trials) from step 1, or 1 / ||g|| before
// the first pair exists; a pair is stored only if s^T y > 1e-12 ||s|| ||y||.
// The vector algebra runs on the device; only scalars come back.
static bfc_status lbfgs_impl(Ctx* c, int iters, int m, bfc_sweep_stats* history, int cap, int32_t* done)
{
    const int64_t M = 2 * c->Pn;  // doubles
    const size_t vb = (size_t)M * sizeof(double);
    std::vector<double*> S(m, nullptr), Y(m, nullptr);
    double *x = nullptr, *g = nullptr, *d = nullptr, *xt = nullptr, *gt = nullptr;
    std::vector<void*> bufs;
    auto get = [&](double** p) -> bfc_status {
        BFC_TRY(dalloc(c, (void**)p, vb, "L-BFGS vectors"));
        bufs.push_back(*p);
        return BFC_OK;
    };
    bfc_status st = BFC_OK;
    for (auto** p : {&x, &g, &d, &xt, &gt})
        if (st == BFC_OK) st = get(p);
    for (int q = 0; q < m && st == BFC_OK; ++q) {
        st = get(&S[q]);
        if (st == BFC_OK) st = get(&Y[q]);
    }
    auto release = [&]() {
        cudaStreamSynchronize(c->stream);
        for (void* p : bufs) dfree(c, p);
    };
    if (st != BFC_OK) { release(); return st; }
    std::vector<double> rho(m, 0.0), alpha(m, 0.0);
    int npairs = 0, head = 0;  // ring buffer of pairs: newest at (head - 1) mod m
    double hs[3];
    const double lam = c->P.lambda;
    auto objective = [&](const double* h) { return 0.5 * h[0] + 0.5 * lam * h[2]; };
    // training-value norm for the relative error
    double tnorm2 = 0.0;
    launch_sumsq(c->d_t, c->N, c->d_red, 1, c->stream);
    st = cudaMemcpyAsync(&tnorm2, c->d_red, sizeof(double), cudaMemcpyDeviceToHost, c->stream) == cudaSuccess
             ? sync(c) : fail(c, BFC_ECUDA, "copy");
    if (st == BFC_OK) st = cudaMemcpyAsync(x, c->z1d, vb, cudaMemcpyDeviceToDevice, c->stream) == cudaSuccess
                               ? BFC_OK : fail(c, BFC_ECUDA, "copy");
    if (st == BFC_OK) st = grad_into(c, 1, (double2*)g, hs);
    double f = objective(hs);
    int k = 0;
    for (; k < iters && st == BFC_OK; ++k) {
        BFC_CK(c, cudaEventRecord(c->ev0, c->stream));
        // two-loop recursion: d = -H g
        BFC_CK(c, cudaMemcpyAsync(d, g, vb, cudaMemcpyDeviceToDevice, c->stream));
        for (int q = 0; q < npairs && st == BFC_OK; ++q) {
            const int idx = ((head - 1 - q) % m + m) % m;
            double sq;
            st = ddot(c, S[idx], d, M, &sq);
            alpha[idx] = rho[idx] * sq;
            launch_axpy(d, Y[idx], -alpha[idx], M, c->stream);
        }
        double gamma = 1.0;
        if (npairs > 0 && st == BFC_OK) {
            const int idx = ((head - 1) % m + m) % m;
            double yy;
            st = ddot(c, Y[idx], Y[idx], M, &yy);
            gamma = 1.0 / (rho[idx] * yy);
        }
        launch_axpby(d, gamma, d, 0.0, d, M, c->stream);
        for (int q = npairs - 1; q >= 0 && st == BFC_OK; --q) {
            const int idx = ((head - 1 - q) % m + m) % m;
            double yr;
            st = ddot(c, Y[idx], d, M, &yr);
            launch_axpy(d, S[idx], alpha[idx] - rho[idx] * yr, M, c->stream);
        }
        launch_axpby(d, -1.0, d, 0.0, d, M, c->stream);
        double gtd = 0.0, gg = 0.0;
        if (st == BFC_OK) st = ddot(c, g, d, M, &gtd);
        if (st == BFC_OK) st = ddot(c, g, g, M, &gg);
        if (st != BFC_OK) break;
        if (!(gtd < 0.0)) {  // not a descent direction: fall back to steepest descent
            launch_axpby(d, -1.0, g, 0.0, g, M, c->stream);
            gtd = -gg;
        }
        double step = (npairs == 0 && k == 0) ? 1.0 / std::sqrt(gg) : 1.0;
        double ft = f;
        for (int ls = 0; ls < 30 && st == BFC_OK; ++ls) {
            launch_axpby(xt, 1.0, x, step, d, M, c->stream);
            BFC_CK(c, cudaMemcpyAsync(c->z1d, xt, vb, cudaMemcpyDeviceToDevice, c->stream));
            st = refresh_copies(c);
            if (st == BFC_OK) st = grad_into(c, 1, (double2*)gt, hs);
            ft = objective(hs);
            if (ft <= f + 1e-4 * step * gtd) break;
            step *= 0.5;
        }
        if (st != BFC_OK) break;
        // new pair s = xt - x, y = gt - g
        const int slot = head;
        launch_axpby(S[slot], 1.0, xt, -1.0, x, M, c->stream);
        launch_axpby(Y[slot], 1.0, gt, -1.0, g, M, c->stream);
        double sy = 0.0, ss = 0.0, yy = 0.0;
        st = ddot(c, S[slot], Y[slot], M, &sy);
        if (st == BFC_OK) st = ddot(c, S[slot], S[slot], M, &ss);
        if (st == BFC_OK) st = ddot(c, Y[slot], Y[slot], M, &yy);
        if (st != BFC_OK) break;
        if (sy > 1e-12 * std::sqrt(ss) * std::sqrt(yy)) {
            rho[slot] = 1.0 / sy;
            head = (head + 1) % m;
            npairs = std::min(npairs + 1, m);
        }
        std::swap(x, xt);
        std::swap(g, gt);
        f = ft;
        if (c->NT > 0) {
            st = test_error(c, 3);
            if (st == BFC_OK) st = sync(c);
        }
        BFC_CK(c, cudaEventRecord(c->ev1, c->stream));
        double th[2] = {0.0, 1.0};
        if (c->NT > 0) BFC_CK(c, cudaMemcpyAsync(th, c->d_scalars + 3, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (st == BFC_OK) st = sync(c);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        if (history && k < cap) {
            bfc_sweep_stats& h = history[k];
            memset(&h, 0, sizeof(h));
            h.sweep = k + 1;
            h.train_rel_err = tnorm2 > 0 ? std::sqrt(hs[0] / tnorm2) : std::sqrt(hs[0]);
            h.test_rel_err = c->NT > 0 ? (th[1] > 0 ? std::sqrt(th[0] / th[1]) : std::sqrt(th[0])) : -1.0;
            h.objective = f;
            h.sweep_ms = ms;
            h.entries_per_s = ms > 0 ? (double)c->N / (ms * 1e-3) : 0.0;
        }
    }
    if (done) *done = k;
    // the factors hold the last evaluated point; make them the accepted one
    if (st == BFC_OK) {
        if (cudaMemcpyAsync(c->z1d, x, vb, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            st = fail(c, BFC_ECUDA, "copy");
        if (st == BFC_OK) st = refresh_copies(c);
    }
    release();
    if (st == BFC_OK) st = sync(c);
    return st;
}

bool level_grouped(const Ctx* c, int m)
{
    if (c->P.gram_impl != 0 || (c->r != 4 && c->r != 8) || !c->grec) return false;
    if (m < 1 || m > c->L || (int)c->grp.size() <= m) return false;
    const GroupLevel& gl = c->grp[m];
    if (!gl.gstart) return false;   // level order not grouped at build time
    const double ratio = c->gram_tc ? c->grp_max_ratio : c->grp_cuda_ratio;
    return gl.ngroups > 0 && (double)gl.ngroups < ratio * (double)c->N;
}

}  // namespace bfc

using namespace bfc;

// ==================================================================== ABI

extern "C" {

int64_t bfc_num_params(int64_t n, int32_t L, int32_t b, int32_t r)
{
    if (L < 0 || L > 24 || b < 1 || r < 1 || n != (int64_t)b << L) return -1;
    return 2 * n * r + (int64_t)L * ((int64_t)1 << (L + 1)) * r * r;
}

bfc_status bfc_create(const bfc_params* params, int64_t nnz, const int32_t* i, const int32_t* j, const double* t,
                      int64_t ntest, const int32_t* it, const int32_t* jt, const double* tt, bfc_ctx** out)
{
    Inputs in{nnz, i, j, t, ntest, it, jt, tt,
              (params && params->values_on_device) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice};
    return create_impl(params, in, out);
}

bfc_status bfc_set_stream(bfc_ctx* ctx, void* cuda_stream)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    BFC_TRY(sync(c));
    c->stream = cuda_stream ? (cudaStream_t)cuda_stream : c->own_stream;
    return BFC_OK;
}

bfc_status bfc_set_factors(bfc_ctx* ctx, const double* packed)
{
    Ctx* c = (Ctx*)ctx;
    if (!c || !packed) return c ? fail(c, BFC_EINVAL, "null factors") : BFC_EINVAL;
    BFC_CK(c, cudaMemcpyAsync(c->z1d, packed, (size_t)c->Pn * 16, in_kind(c), c->stream));
    BFC_TRY(refresh_copies(c));
    return sync(c);
}

bfc_status bfc_get_factors(bfc_ctx* ctx, double* packed)
{
    Ctx* c = (Ctx*)ctx;
    if (!c || !packed) return c ? fail(c, BFC_EINVAL, "null output") : BFC_EINVAL;
    BFC_CK(c, cudaMemcpyAsync(packed, c->z1d, (size_t)c->Pn * 16, out_kind(c), c->stream));
    return sync(c);
}

bfc_status bfc_eval(bfc_ctx* ctx, int64_t m, const int32_t* i, const int32_t* j, double* out)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    if (m < 0 || (m > 0 && (!i || !j || !out))) return fail(c, BFC_EINVAL, "bad eval arguments");
    if (m == 0) return BFC_OK;
    const size_t ib = ((size_t)m * 4 + 255) / 256 * 256;
    BFC_TRY(ensure_tmp(c, 2 * ib + (size_t)m * 16 + 256));
    int32_t* di = (int32_t*)c->d_tmp;
    int32_t* dj = (int32_t*)((char*)c->d_tmp + ib);
    double2* dout = (double2*)((char*)c->d_tmp + 2 * ib);
    BFC_CK(c, cudaMemcpyAsync(di, i, m * 4, in_kind(c), c->stream));
    BFC_CK(c, cudaMemcpyAsync(dj, j, m * 4, in_kind(c), c->stream));
    int* dflag = (int*)(c->d_count + 4);
    BFC_CK(c, cudaMemsetAsync(dflag, 0, sizeof(int), c->stream));
    launch_check_entries(di, dj, nullptr, m, c->n, dflag, c->stream);
    int hflag = 0;
    BFC_CK(c, cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    BFC_TRY(sync(c));
    if (hflag) return fail(c, BFC_EINVAL, "an index is outside [0, n)");
    const Ops* ops = get_ops(c->fp32, c->r);
    const int nb = (int)std::min<int64_t>(1216 * 4, (m + 255) / 256);
    BFC_TRY(ops->eval(c, di, dj, m, dout, nullptr, nullptr, nb));
    BFC_CK(c, cudaMemcpyAsync(out, dout, (size_t)m * 16, out_kind(c), c->stream));
    return sync(c);
}

bfc_status bfc_als_sweep(bfc_ctx* ctx, bfc_sweep_stats* out)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    return sweep_impl(c, out, true);
}

bfc_status bfc_grad(bfc_ctx* ctx, int32_t include_reg, double* grad_packed, double* objective)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    const size_t gb = (size_t)c->Pn * 16;
    BFC_TRY(ensure_tmp(c, gb + 256));
    double2* G = (double2*)c->d_tmp;
    double hs[3];
    BFC_TRY(grad_into(c, include_reg, G, hs));
    if (grad_packed) {
        BFC_CK(c, cudaMemcpyAsync(grad_packed, G, gb, out_kind(c), c->stream));
        BFC_TRY(sync(c));
    }
    if (objective) *objective = 0.5 * hs[0] + (include_reg ? 0.5 * c->P.lambda * hs[2] : 0.0);
    return BFC_OK;
}

bfc_status bfc_lbfgs(bfc_ctx* ctx, int32_t iters, int32_t memory, bfc_sweep_stats* history, int32_t history_cap,
                     int32_t* done)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    if (done) *done = 0;
    if (iters < 0 || memory < 1 || memory > 64) return fail(c, BFC_EINVAL, "iters >= 0 and 1 <= memory <= 64 required");
    return lbfgs_impl(c, iters, memory, history, history_cap, done);
}

// Alg. 2 on device A, B (n x R) with host or device Gaussians (gkind) into
// the context's FP64 factors; the compute copies are refreshed.
static bfc_status lr2bf_into(Ctx* c, int R, const double2* A, const double2* B, const double* gauss,
                             cudaMemcpyKind gkind, int p)
{
    const int64_t gcount = lr2bf_gaussian_count(c->n, c->L, c->b, c->r, p);
    const size_t gb = ((size_t)gcount * 16 + 255) / 256 * 256;
    const size_t sb = lr2bf_scratch_bytes(c->n, c->L, c->b, R, c->r, p);
    BFC_TRY(ensure_tmp(c, gb + sb));
    double2* G = (double2*)c->d_tmp;
    BFC_CK(c, cudaMemcpyAsync(G, gauss, (size_t)gcount * 16, gkind, c->stream));
    cudaError_t e = lr2bf_run(A, B, G, c->n, c->L, c->b, R, c->r, p, c->z1d, c->Zd, c->zLd, (char*)c->d_tmp + gb,
                              c->stream);
    if (e != cudaSuccess) return fail(c, BFC_ECUDA, std::string("low-rank to butterfly: ") + cudaGetErrorString(e));
    BFC_TRY(refresh_copies(c));
    return sync(c);
}

// Low-rank start: rank-R completion (Alg. 1 with L = 0) from A0, B0, then the
// exact embedding (gauss == nullptr) or Alg. 2 with the given host Gaussians.
static bfc_status lowrank_init_impl(Ctx* c, int32_t R, int32_t sweeps, const double* A0, const double* B0,
                                    const double* gauss, int p)
{
    if (R < 1 || R > c->r || sweeps < 0 || !A0 || !B0) return fail(c, BFC_EINVAL, "bad low-rank arguments");
    // Low-rank completion is Alg. 1 with L = 0 and leaf size n on the same data.
    bfc_params lp = c->P;
    lp.L = 0;
    lp.b = (int32_t)c->n;
    lp.r = R;
    lp.values_on_device = 1;
    Inputs in{c->N, c->d_i, c->d_j, (const double*)c->d_t, 0, nullptr, nullptr, nullptr, cudaMemcpyDeviceToDevice};
    bfc_ctx* lr = nullptr;
    bfc_status st = create_impl(&lp, in, &lr);
    if (st != BFC_OK) return fail(c, st, std::string("low-rank context: ") + g_create_err);
    Ctx* lc = (Ctx*)lr;
    const size_t half = (size_t)c->n * R * 16;
    cudaError_t e1 = cudaMemcpyAsync(lc->z1d, A0, half, in_kind(c), lc->stream);
    cudaError_t e2 = cudaMemcpyAsync(lc->zLd, B0, half, in_kind(c), lc->stream);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        bfc_destroy(lr);
        return fail(c, BFC_ECUDA, "copy of the low-rank start failed");
    }
    st = refresh_copies(lc);
    for (int s = 0; s < sweeps && st == BFC_OK; ++s) st = sweep_impl(lc, nullptr);
    if (st == BFC_OK) st = sync(lc);
    if (st != BFC_OK) {
        std::string m = lc->err;
        bfc_destroy(lr);
        return fail(c, st, "low-rank completion: " + m);
    }
    if (gauss) {
        // Alg. 2 reads lc's factors on c->stream (lr2bf_into synchronizes)
        st = lr2bf_into(c, R, lc->z1d, lc->zLd, gauss, cudaMemcpyHostToDevice, p);
        bfc_destroy(lr);
        return st;
    }
    launch_embed(lc->z1d, lc->zLd, c->n, R, c->r, (int64_t)c->L * c->S, c->z1d, c->Zd, c->zLd, c->stream);
    cudaError_t e = cudaGetLastError();
    // the embedding reads lc's buffers on c->stream: finish before freeing lc
    cudaStreamSynchronize(c->stream);
    bfc_destroy(lr);
    if (e != cudaSuccess) return fail(c, BFC_ECUDA, std::string("embed: ") + cudaGetErrorString(e));
    BFC_TRY(refresh_copies(c));
    return sync(c);
}

bfc_status bfc_lowrank_init(bfc_ctx* ctx, int32_t R, int32_t sweeps, const double* A0, const double* B0)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    return lowrank_init_impl(c, R, sweeps, A0, B0, nullptr, 0);
}

bfc_status bfc_lowrank_to_butterfly(bfc_ctx* ctx, int32_t R, const double* A, const double* B, int32_t p,
                                    const double* gaussians)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    if (R < 1 || R > c->r || p < 0 || c->r + p > 32 || !A || !B || !gaussians)
        return fail(c, BFC_EINVAL, "low-rank to butterfly needs 1 <= R <= r, p >= 0, r + p <= 32 and all arrays");
    if (c->P.values_on_device)
        return lr2bf_into(c, R, (const double2*)A, (const double2*)B, gaussians, cudaMemcpyDeviceToDevice, p);
    // host A, B: staged in a device buffer of the context's own
    double2* AB = nullptr;
    const size_t half = (size_t)c->n * R * 16;
    BFC_TRY(dalloc(c, (void**)&AB, 2 * half, "low-rank factors"));
    BFC_CK(c, cudaMemcpyAsync(AB, A, half, cudaMemcpyHostToDevice, c->stream));
    BFC_CK(c, cudaMemcpyAsync((char*)AB + half, B, half, cudaMemcpyHostToDevice, c->stream));
    const bfc_status st = lr2bf_into(c, R, AB, (const double2*)((char*)AB + half), gaussians,
                                     cudaMemcpyHostToDevice, p);
    cudaStreamSynchronize(c->stream);
    dfree(c, AB);
    return st;
}

// SplitMix64 (Steele, Lea, Flood 2014) + Box-Muller CN(0, sigma^2) start, the
// same published recipe as the seeded input generators.
static void splitmix_cnormal(uint64_t seed, uint64_t& k, int64_t count, double sigma, std::vector<double>& out)
{
    auto next = [&](void) {
        k += 1;
        uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto unif = [&](void) { return ((double)(next() >> 11) + 1.0) * (1.0 / 9007199254740992.0); };
    const int64_t half = count;  // 2*count normals, Box-Muller pairs
    std::vector<double> u1(half), u2(half);
    for (int64_t q = 0; q < half; ++q) u1[q] = unif();
    for (int64_t q = 0; q < half; ++q) u2[q] = unif();
    out.resize(2 * count);
    const double sc = sigma / sqrt(2.0);
    for (int64_t q = 0; q < half; ++q) {
        const double rad = sqrt(-2.0 * log(u1[q]));
        out[2 * q] = rad * cos(2.0 * M_PI * u2[q]) * sc;
        out[2 * q + 1] = rad * sin(2.0 * M_PI * u2[q]) * sc;
    }
}

// Start of the full workflow: the optional low-rank start (init_kind 1).
static bfc_status complete_init(Ctx* c)
{
    if (c->P.init_kind == 1 || c->P.init_kind == 2) {
        const int R = c->P.lr_rank > 0 ? c->P.lr_rank : c->r;
        if (R > c->r) return fail(c, BFC_EINVAL, "lr_rank > r");
        // rms of the training values
        launch_sumsq(c->d_t, c->N, c->d_red, 1, c->stream);
        double ss = 0.0;
        BFC_CK(c, cudaMemcpyAsync(&ss, c->d_red, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        BFC_TRY(sync(c));
        const double rms = sqrt(ss / (double)c->N);
        const double sigma = sqrt(rms / R);
        uint64_t k = 0;
        std::vector<double> A, B;
        splitmix_cnormal(c->P.seed, k, c->n * R, sigma, A);
        splitmix_cnormal(c->P.seed, k, c->n * R, sigma, B);
        // init_kind 2: Alg. 2's Gaussians from a second SplitMix64 stream,
        // seed params.seed + 1, CN(0, 1), in the order the conversion reads them
        std::vector<double> G;
        const int p = c->P.lr2bf_oversample > 0 ? c->P.lr2bf_oversample : 5;
        if (c->P.init_kind == 2) {
            if (c->r + p > 32) return fail(c, BFC_EINVAL, "r + lr2bf_oversample must be <= 32");
            uint64_t kg = 0;
            splitmix_cnormal(c->P.seed + 1, kg, lr2bf_gaussian_count(c->n, c->L, c->b, c->r, p), 1.0, G);
        }
        const int32_t saved = c->P.values_on_device;
        c->P.values_on_device = 0;
        bfc_status st = lowrank_init_impl(c, R, c->P.lr_sweeps, A.data(), B.data(),
                                          c->P.init_kind == 2 ? G.data() : nullptr, p);
        c->P.values_on_device = saved;
        BFC_TRY(st);
    }
    return BFC_OK;
}

// Relative error ||x - t|| / ||t|| of the current factors over the training
// entries (Eq. (BF_convergence)), through d_scalars[12..13].
static bfc_status train_rel_err(Ctx* c, double* err)
{
    const Ops* ops = get_ops(c->fp32, c->r);
    const int nb = (int)std::min<int64_t>(1216, (c->N + 255) / 256);
    BFC_TRY(ops->eval(c, c->d_i, c->d_j, c->N, nullptr, c->d_t, c->d_red, nb));
    launch_reduce_pairs(c->d_red, nb, c->d_scalars + 12, c->stream);
    BFC_LAUNCH_CHECK(c, "reduce");
    double hs[2];
    BFC_CK(c, cudaMemcpyAsync(hs, c->d_scalars + 12, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    BFC_TRY(sync(c));
    *err = hs[1] > 0 ? sqrt(hs[0] / hs[1]) : sqrt(hs[0]);
    return BFC_OK;
}

// End of the full workflow in the precision form: params.refine_sweeps
// sweeps of the FP64 path from the current factors, in a child context on
// the same data; the factors come back into this context.  Stats of each
// sweep go to history[*done ...].
static bfc_status complete_refine(Ctx* c, bfc_sweep_stats* history, int32_t history_cap, int32_t* done)
{
    if (!c->fp32 || c->P.refine_sweeps <= 0) return BFC_OK;
    bfc_params fp = c->P;
    fp.prec = BFC_PREC_FP64;
    fp.values_on_device = 1;
    fp.init_kind = 0;
    fp.refine_sweeps = 0;
    Inputs in{c->N, c->d_i, c->d_j, (const double*)c->d_t, c->NT, c->d_it, c->d_jt, (const double*)c->d_tt,
              cudaMemcpyDeviceToDevice};
    BFC_TRY(sync(c));
    bfc_ctx* child = nullptr;
    bfc_status st = create_impl(&fp, in, &child);
    if (st != BFC_OK) return fail(c, st, std::string("FP64 refinement context: ") + g_create_err);
    Ctx* fc = (Ctx*)child;
    cudaError_t e = cudaMemcpyAsync(fc->z1d, c->z1d, (size_t)c->Pn * 16, cudaMemcpyDeviceToDevice, fc->stream);
    if (e != cudaSuccess) st = fail(c, BFC_ECUDA, std::string("refinement copy: ") + cudaGetErrorString(e));
    for (int s = 0; s < c->P.refine_sweeps && st == BFC_OK; ++s) {
        bfc_sweep_stats rs{};
        st = sweep_impl(fc, &rs);
        if (st != BFC_OK) {
            st = fail(c, st, "FP64 refinement sweep: " + fc->err);
            break;
        }
        c->sweeps_done += 1;
        rs.sweep = c->sweeps_done;
        if (history && *done < history_cap) history[*done] = rs;
        ++*done;
    }
    if (st == BFC_OK) st = sync(fc);
    if (st == BFC_OK) {
        e = cudaMemcpyAsync(c->z1d, fc->z1d, (size_t)c->Pn * 16, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = fail(c, BFC_ECUDA, std::string("refinement copy back: ") + cudaGetErrorString(e));
    }
    bfc_destroy(child);
    BFC_TRY(st);
    BFC_TRY(refresh_copies(c));
    return sync(c);
}

bfc_status bfc_complete(bfc_ctx* ctx, bfc_sweep_stats* history, int32_t history_cap, int32_t* nsweeps)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    if (nsweeps) *nsweeps = 0;
    BFC_TRY(complete_init(c));
    int done = 0;
    for (int s = 0; s < c->P.max_sweeps; ++s) {
        bfc_sweep_stats st{};
        BFC_TRY(sweep_impl(c, &st, true));
        if (history && done < history_cap) history[done] = st;
        ++done;
        if (st.train_rel_err < c->P.tol) break;
    }
    bfc_status st = complete_refine(c, history, history_cap, &done);
    if (nsweeps) *nsweeps = done;
    return st;
}

}  // extern "C"

// Statistics of one first-order iteration: the training residual partials
// (per column fiber in d_red) are reduced, ||S||^2 and the test error added.
static bfc_status fo_iter_stats(Ctx* c, bfc_sweep_stats* out, int64_t launched0)
{
    {
        ProfScope ps(c, "reduce");
        launch_reduce_pairs(c->d_red, c->n, c->d_scalars + 0, c->stream);
    }
    BFC_LAUNCH_CHECK(c, "reduce");
    BFC_TRY(factor_sumsq(c, 2));
    BFC_TRY(test_error(c, 3));
    BFC_CK(c, cudaEventRecord(c->ev1, c->stream));
    c->sweeps_done += 1;
    BFC_TRY(sync(c));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    BFC_TRY(collect_stats(c, out, ms));
    out->launches = c->n_launch - launched0;
    out->gram_impl = -1;
    return BFC_OK;
}

// Runs `iters` iterations of a first-order method (one_iter enqueues one),
// recording statistics and stopping early once the training error is below
// params.tol.
template <typename F>
static bfc_status fo_run(Ctx* c, int32_t iters, bfc_sweep_stats* history, int32_t cap, int32_t* done, F one_iter)
{
    if (done) *done = 0;
    for (int32_t it = 1; it <= iters; ++it) {
        const int64_t l0 = c->n_launch;
        BFC_CK(c, cudaMemsetAsync(c->d_count, 0, 3 * sizeof(unsigned long long), c->stream));
        BFC_CK(c, cudaEventRecord(c->ev0, c->stream));
        BFC_TRY(one_iter(it));
        bfc_sweep_stats st{};
        BFC_TRY(fo_iter_stats(c, &st, l0));
        st.sweep = it;
        if (history && it <= cap) history[it - 1] = st;
        if (done) *done = it;
        if (st.train_rel_err < c->P.tol) break;
    }
    return BFC_OK;
}

extern "C" {

bfc_status bfc_matvec(bfc_ctx* ctx, int32_t nvec, const double* V, double* U)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    if (nvec < 1 || nvec > 4096 || !V || !U) return fail(c, BFC_EINVAL, "matvec needs 1 <= nvec <= 4096 and vectors");
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t vb = up((size_t)c->n * nvec * 16);
    const size_t yb = up((size_t)c->S * nvec * c->r * c->vsz);
    BFC_TRY(ensure_tmp(c, 2 * vb + 2 * yb));
    char* base = (char*)c->d_tmp;
    double2* Vd = (double2*)base;
    double2* Ud = (double2*)(base + vb);
    void* y0 = base + 2 * vb;
    void* y1 = base + 2 * vb + yb;
    BFC_CK(c, cudaMemcpyAsync(Vd, V, (size_t)c->n * nvec * 16, in_kind(c), c->stream));
    BFC_TRY(get_fo_ops(c->fp32, c->r)->matvec(c, nvec, Vd, Ud, y0, y1));
    BFC_CK(c, cudaMemcpyAsync(U, Ud, (size_t)c->n * nvec * 16, out_kind(c), c->stream));
    return sync(c);
}

bfc_status bfc_adam(bfc_ctx* ctx, int32_t iters, double alpha, double beta1, double beta2, double sigma,
                    bfc_sweep_stats* history, int32_t history_cap, int32_t* done)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    if (done) *done = 0;
    if (iters < 0 || !(alpha > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) ||
        !(sigma >= 0.0))
        return fail(c, BFC_EINVAL, "ADAM needs iters >= 0, alpha > 0, 0 <= beta1, beta2 < 1, sigma >= 0");
    if (!c->adam_m) {
        BFC_TRY(dalloc(c, (void**)&c->adam_m, (size_t)c->Pn * sizeof(double2), "ADAM first moments"));
        BFC_TRY(dalloc(c, (void**)&c->adam_v, (size_t)c->Pn * sizeof(double2), "ADAM second moments"));
    }
    BFC_CK(c, cudaMemsetAsync(c->adam_m, 0, (size_t)c->Pn * sizeof(double2), c->stream));
    BFC_CK(c, cudaMemsetAsync(c->adam_v, 0, (size_t)c->Pn * sizeof(double2), c->stream));
    const FoOps* fo = get_fo_ops(c->fp32, c->r);
    return fo_run(c, iters, history, history_cap, done, [&](int32_t it) {
        AdamHyper hp;
        hp.alpha = alpha;
        hp.beta1 = beta1;
        hp.beta2 = beta2;
        hp.sigma = sigma;
        hp.inv1 = 1.0 / (1.0 - pow(beta1, (double)it));
        hp.inv2 = 1.0 / (1.0 - pow(beta2, (double)it));
        return fo->adam_iter(c, hp, c->adam_m, c->adam_v);
    });
}

bfc_status bfc_adf(bfc_ctx* ctx, int32_t iters, bfc_sweep_stats* history, int32_t history_cap, int32_t* done)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    if (done) *done = 0;
    if (iters < 0) return fail(c, BFC_EINVAL, "iters must be >= 0");
    if ((c->L > 0 && c->b < c->r) || c->n < c->r)
        return fail(c, BFC_EINVAL, "ADF orthogonalizes b x r leaf blocks: needs b >= r");
    const FoOps* fo = get_fo_ops(c->fp32, c->r);
    return fo_run(c, iters, history, history_cap, done, [&](int32_t) { return fo->adf_iter(c); });
}

bfc_status bfc_canonicalize(bfc_ctx* ctx)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    if ((c->L > 0 && c->b < c->r) || c->n < c->r)
        return fail(c, BFC_EINVAL, "the gauge is fixed by QR of b x r leaf blocks: needs b >= r");
    const cudaError_t e = launch_canonicalize(c->z1d, c->Zd, c->zLd, c->n, c->L, c->b, c->r, c->stream);
    if (e != cudaSuccess) return fail(c, BFC_ECUDA, std::string("canonicalize: ") + cudaGetErrorString(e));
    BFC_TRY(refresh_copies(c));
    return sync(c);
}

bfc_status bfc_init_learned(bfc_ctx* ctx, bfc_mlp* model, double omega, double offset, int32_t allow_fallback,
                            int32_t* used_learned, double* start_err)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    if (used_learned) *used_learned = 0;
    if (!model) return fail(c, BFC_EINVAL, "null model");
    int32_t din = 0, dhid = 0;
    int64_t dout = 0;
    bfc_mlp_dims(model, &din, &dhid, &dout);
    if (din != 2 || dout != 2 * c->Pn)
        return fail(c, BFC_EINVAL, "model must map 2 inputs to the 2 P reals of this context's factors");
    if (!isfinite(omega) || !isfinite(offset)) return fail(c, BFC_EINVAL, "omega and offset must be finite");
    const double x[2] = {omega / (M_PI * (double)c->n), offset};
    std::vector<double> y((size_t)dout);
    bfc_status st = bfc_mlp_forward(model, 1, x, y.data());
    if (st != BFC_OK) return fail(c, st, std::string("learned start: ") + bfc_last_error(nullptr));
    for (double v : y)
        if (!isfinite(v)) return fail(c, BFC_ENONFINITE, "learned start is not finite");
    BFC_CK(c, cudaMemcpyAsync(c->z1d, y.data(), (size_t)c->Pn * 16, cudaMemcpyHostToDevice, c->stream));
    BFC_TRY(refresh_copies(c));
    double e_learned = 0.0;
    BFC_TRY(train_rel_err(c, &e_learned));
    if (used_learned) *used_learned = 1;
    if (start_err) *start_err = e_learned;
    if (!allow_fallback) return BFC_OK;
    // the low-rank start remains the fallback: keep whichever fits the
    // training entries better
    const bfc_params saved = c->P;
    c->P.init_kind = 1;
    st = complete_init(c);
    c->P = saved;
    BFC_TRY(st);
    double e_lr = 0.0;
    BFC_TRY(train_rel_err(c, &e_lr));
    if (e_lr < e_learned) {
        if (used_learned) *used_learned = 0;
        if (start_err) *start_err = e_lr;
        return BFC_OK;
    }
    BFC_CK(c, cudaMemcpyAsync(c->z1d, y.data(), (size_t)c->Pn * 16, cudaMemcpyHostToDevice, c->stream));
    BFC_TRY(refresh_copies(c));
    return sync(c);
}

}  // extern "C"

// Batched completion in one launch: per problem, a conditional WHILE graph
// node whose body is the problem's captured sweep followed by k_batch_step,
// which turns the sweep's device scalars into its statistics (the host
// formulas of collect_stats), stores them in the problem's history and
// decides on the device whether the loop goes on (train error >= tol,
// fewer than max_sweeps sweeps, finite residual, no expired device wait).
// The loop count is bounded by max_sweeps.
struct BatchSlot {
    double* hist;      // [max_sweeps][8]: train err, test err, objective, singular, fallbacks, refine steps, wait flag
    int32_t* nsweeps;  // sweeps done by the launch
};

__global__ void k_batch_step(cudaGraphConditionalHandle h, const double* __restrict__ sc,
                             const unsigned long long* __restrict__ cnt, BatchSlot slot, int max_sweeps, double tol,
                             double lambda, int has_test)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int d = *slot.nsweeps;
    const double tr = sc[1] > 0 ? sqrt(sc[0] / sc[1]) : sqrt(sc[0]);
    const double te = has_test ? (sc[4] > 0 ? sqrt(sc[3] / sc[4]) : sqrt(sc[3])) : -1.0;
    double* hr = slot.hist + (size_t)(d < max_sweeps ? d : max_sweeps - 1) * 8;
    hr[0] = tr;
    hr[1] = te;
    hr[2] = 0.5 * sc[0] + 0.5 * lambda * sc[2];
    hr[3] = (double)cnt[0];
    hr[4] = (double)cnt[1];
    hr[5] = (double)cnt[2];
    hr[6] = (double)cnt[5];
    *slot.nsweeps = d + 1;
    const bool go = d + 1 < max_sweeps && !(tr < tol) && isfinite(sc[0]) && cnt[5] == 0;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// Runs the remaining sweeps of the active problems as one graph launch.
// Returns BFC_OK with *ran = false (nothing launched) when the graph cannot
// be built (the caller then runs the sweeps round by round).
static bfc_status batch_one_launch(std::vector<Ctx*>& cs, std::vector<char>& active, std::vector<int>& done,
                                   std::vector<bfc_sweep_stats>& st, bool* ran)
{
    *ran = false;
    const int32_t count = (int32_t)cs.size();
    std::vector<int32_t> rem((size_t)count, 0), off((size_t)count + 1, 0);
    for (int32_t q = 0; q < count; ++q) {
        rem[q] = active[q] ? std::max(cs[q]->P.max_sweeps - done[q], 0) : 0;
        if (rem[q] > 0 && !cs[q]->sweep_graph_src) return BFC_OK;
        off[q + 1] = off[q] + rem[q];
    }
    if (off[count] == 0) return BFC_OK;
    double* dh = nullptr;
    int32_t* dn = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaStream_t bs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
        if (bs) cudaStreamDestroy(bs);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (dh) cudaFree(dh);
        if (dn) cudaFree(dn);
    };
    cudaError_t e = cudaMalloc(&dh, (size_t)off[count] * 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dn, (size_t)count * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(dn, 0, (size_t)count * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) {
        cleanup();
        return fail(nullptr, BFC_ECUDA, std::string("batch launch set-up: ") + cudaGetErrorString(e));
    }
    // graph construction: a failure here leaves the rounds to the caller
    bool built = true;
    for (int32_t q = 0; q < count && built; ++q) {
        if (rem[q] == 0) continue;
        Ctx* c = cs[q];
        cudaGraphConditionalHandle h;
        built = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cn = nullptr;
        if (built) built = cudaGraphAddNode(&cn, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
        if (!built) break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaGraphNode_t sweep = nullptr, step = nullptr;
        built = cudaGraphAddChildGraphNode(&sweep, body, nullptr, 0, c->sweep_graph_src) == cudaSuccess;
        BatchSlot slot{dh + (size_t)off[q] * 8, dn + q};
        int maxs = rem[q];
        double tol = c->P.tol, lam = c->P.lambda;
        int has_test = c->NT > 0 ? 1 : 0;
        const double* sc = c->d_scalars;
        const unsigned long long* cnt = c->d_count;
        void* args[] = {&h, &sc, &cnt, &slot, &maxs, &tol, &lam, &has_test};
        cudaKernelNodeParams kp = {};
        kp.func = (void*)k_batch_step;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(32);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        if (built) built = cudaGraphAddKernelNode(&step, body, &sweep, 1, &kp) == cudaSuccess;
    }
    if (built) built = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
    if (!built) {
        cudaGetLastError();
        cleanup();
        return BFC_OK;
    }
    e = cudaEventRecord(e0, bs);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, bs);
    if (e == cudaSuccess) e = cudaEventRecord(e1, bs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(bs);
    std::vector<double> hh((size_t)off[count] * 8);
    std::vector<int32_t> hn((size_t)count);
    if (e == cudaSuccess) e = cudaMemcpy(hh.data(), dh, hh.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hn.data(), dn, hn.size() * sizeof(int32_t), cudaMemcpyDeviceToHost);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cleanup();
    if (e != cudaSuccess) return fail(nullptr, BFC_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    *ran = true;
    int32_t rounds = 1;
    for (int32_t q = 0; q < count; ++q) rounds = std::max(rounds, hn[q]);
    for (int32_t q = 0; q < count; ++q) {
        if (rem[q] == 0) continue;
        Ctx* c = cs[q];
        const int32_t d = std::min(hn[q], rem[q]);
        c->sweeps_done += d;
        c->n_launch += (int64_t)d * (c->graph_launches + 1);
        done[q] += d;
        active[q] = 0;
        if (d <= 0) continue;
        const double* hr = hh.data() + (size_t)(off[q] + d - 1) * 8;
        bfc_sweep_stats& o = st[q];
        o.sweep = c->sweeps_done;
        o.train_rel_err = hr[0];
        o.test_rel_err = hr[1];
        o.objective = hr[2];
        o.sweep_ms = ms / rounds;   // the launch's time per round of sweeps
        o.entries_per_s = o.sweep_ms > 0 ? (double)c->N / (o.sweep_ms * 1e-3) : 0.0;
        o.singular_slices = (int64_t)hr[3];
        o.refined_fallbacks = (int64_t)hr[4];
        o.refine_steps = (int64_t)hr[5];
        o.launches = (int64_t)d * (c->graph_launches + 1);
        o.gram_impl = c->fp32 ? (c->gram_tc ? 0 : 1) : -1;
        o.batch_launches = 1;
        if (hr[6] != 0.0) {
            cudaMemsetAsync(c->d_count + 5, 0, sizeof(unsigned long long), c->stream);
            sync(c);
            return fail(c, BFC_ETIMEOUT, "a bounded device wait expired (tensor-core Gram or bulk copy)");
        }
        if (!isfinite(hr[0])) return fail(c, BFC_ENONFINITE, "training residual is not finite");
    }
    return BFC_OK;
}

extern "C" {

bfc_status bfc_batch_complete(int32_t count, bfc_ctx* const* ctxs, bfc_sweep_stats* last)
{
    if (count < 0 || (count > 0 && !ctxs)) return fail(nullptr, BFC_EINVAL, "bad batch arguments");
    std::vector<Ctx*> cs((size_t)count);
    for (int32_t q = 0; q < count; ++q) {
        cs[q] = (Ctx*)ctxs[q];
        if (!cs[q]) return fail(nullptr, BFC_EINVAL, "null context in the batch");
        for (int32_t p = 0; p < q; ++p)
            if (cs[p] == cs[q]) return fail(nullptr, BFC_EINVAL, "a context appears twice in the batch");
    }
    auto bad = [&](Ctx* c, bfc_status st) {
        g_create_err = "batch: " + c->err;
        return st;
    };
    std::vector<bfc_sweep_stats> st((size_t)count);
    std::vector<int> done((size_t)count, 0);
    std::vector<char> active((size_t)count, 1);
    for (int32_t q = 0; q < count; ++q) {
        const bfc_status s0 = complete_init(cs[q]);
        if (s0 != BFC_OK) return bad(cs[q], s0);
        if (cs[q]->P.max_sweeps <= 0) active[q] = 0;
    }
    auto stop = [&](int32_t q) {
        return st[q].train_rel_err < cs[q]->P.tol || done[q] >= cs[q]->P.max_sweeps;
    };
    // Autotune the middle-level Gram kernel per rank in the precision form
    // (gram_impl 0: tensor cores unless the CUDA-core kernel is faster on
    // this batch): on the first problem of each rank, one warm-up and one
    // timed sweep with each kernel; the faster serves every problem of that
    // rank.  The four sweeps are ordinary ALS sweeps of that problem.
    for (int r = 1; r <= 8; ++r) {
        int32_t q0 = -1;
        for (int32_t q = 0; q < count; ++q)
            if (cs[q]->fp32 && cs[q]->r == r && cs[q]->P.gram_impl == 0 && active[q]) { q0 = q; break; }
        if (q0 < 0 || cs[q0]->P.max_sweeps < 4) continue;
        Ctx* c = cs[q0];
        float ms[2] = {0.f, 0.f};
        for (int trial = 0; trial < 4 && active[q0]; ++trial) {
            c->gram_tc = (trial & 1) == 0;
            const bfc_status s1 = sweep_impl(c, &st[q0]);
            if (s1 != BFC_OK) return bad(c, s1);
            done[q0] += 1;
            if (trial >= 2) ms[trial & 1] = (float)st[q0].sweep_ms;
            if (stop(q0)) active[q0] = 0;
        }
        const bool tc = !(ms[1] > 0.f && ms[0] > 0.f && ms[1] < ms[0]);
        for (int32_t q = 0; q < count; ++q)
            if (cs[q]->fp32 && cs[q]->r == r && cs[q]->P.gram_impl == 0) cs[q]->gram_tc = tc;
    }
    // rounds: the sweeps of all active problems are the child graphs of one
    // graph, launched once per round (the problems run concurrently); the
    // graph is rebuilt only when the set of active problems changes.  A
    // problem without a captured sweep (profiling on) runs on its own stream.
    for (int32_t q = 0; q < count; ++q)
        if (active[q]) {
            const bfc_status s2 = capture_sweep(cs[q]);
            if (s2 != BFC_OK) return bad(cs[q], s2);
        }
    // all remaining sweeps as one launch (conditional WHILE nodes); the
    // rounds below run only where that graph cannot be built
    {
        bool ran = false;
        const bfc_status sl = batch_one_launch(cs, active, done, st, &ran);
        if (sl != BFC_OK) return sl;
    }
    int32_t nrounds = 0;
    cudaStream_t bs = nullptr;
    cudaGraphExec_t round = nullptr;
    std::vector<char> round_set;
    auto cleanup = [&](void) {
        if (round) cudaGraphExecDestroy(round);
        if (bs) cudaStreamDestroy(bs);
        round = nullptr;
        bs = nullptr;
    };
    if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess)
        return fail(nullptr, BFC_ECUDA, "batch stream");
    for (;;) {
        bool any = false, all_graphs = true;
        for (int32_t q = 0; q < count; ++q)
            if (active[q]) {
                any = true;
                all_graphs = all_graphs && cs[q]->sweep_graph_src != nullptr;
            }
        if (!any) break;
        ++nrounds;
        if (all_graphs) {
            std::vector<char> want(active.begin(), active.end());
            if (!round || want != round_set) {
                if (round) cudaGraphExecDestroy(round);
                round = nullptr;
                cudaGraph_t g = nullptr;
                cudaError_t e = cudaGraphCreate(&g, 0);
                for (int32_t q = 0; q < count && e == cudaSuccess; ++q) {
                    if (!active[q]) continue;
                    Ctx* c = cs[q];
                    cudaGraphNode_t n0 = nullptr, nc = nullptr, n1 = nullptr;
                    e = cudaGraphAddEventRecordNode(&n0, g, nullptr, 0, c->ev0);
                    if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&nc, g, &n0, 1, c->sweep_graph_src);
                    if (e == cudaSuccess) e = cudaGraphAddEventRecordNode(&n1, g, &nc, 1, c->ev1);
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&round, g, 0);
                if (g) cudaGraphDestroy(g);
                if (e != cudaSuccess) {
                    cleanup();
                    return fail(nullptr, BFC_ECUDA, std::string("batch round graph: ") + cudaGetErrorString(e));
                }
                round_set = want;
            }
            cudaError_t e = cudaGraphLaunch(round, bs);
            if (e == cudaSuccess) e = cudaStreamSynchronize(bs);
            if (e != cudaSuccess) {
                cleanup();
                return fail(nullptr, BFC_ECUDA, std::string("batch round: ") + cudaGetErrorString(e));
            }
            for (int32_t q = 0; q < count; ++q)
                if (active[q]) cs[q]->n_launch += cs[q]->graph_launches;
        } else {
            for (int32_t q = 0; q < count; ++q) {
                if (!active[q]) continue;
                Ctx* c = cs[q];
                if (cudaEventRecord(c->ev0, c->stream) != cudaSuccess) {
                    cleanup();
                    return bad(c, fail(c, BFC_ECUDA, "event"));
                }
                const bfc_status s3 = sweep_enqueue(c);
                if (s3 != BFC_OK || cudaEventRecord(c->ev1, c->stream) != cudaSuccess) {
                    cleanup();
                    return bad(c, s3 != BFC_OK ? s3 : fail(c, BFC_ECUDA, "event"));
                }
            }
        }
        for (int32_t q = 0; q < count; ++q) {
            if (!active[q]) continue;
            Ctx* c = cs[q];
            const bfc_status s4 = sweep_finish(c, &st[q], c->sweep_graph ? c->graph_launches : 0);
            if (s4 != BFC_OK) {
                cleanup();
                return bad(c, s4);
            }
            done[q] += 1;
            st[q].batch_launches = nrounds;
            if (stop(q)) active[q] = 0;
        }
    }
    cleanup();
    for (int32_t q = 0; q < count; ++q) {
        int32_t d = 0;
        std::vector<bfc_sweep_stats> rs((size_t)std::max(cs[q]->P.refine_sweeps, 1));
        const bfc_status s5 = complete_refine(cs[q], rs.data(), (int32_t)rs.size(), &d);
        if (s5 != BFC_OK) return bad(cs[q], s5);
        if (d > 0) st[q] = rs[d - 1];   // the last FP64 refinement sweep
        if (last) last[q] = st[q];
    }
    return BFC_OK;
}

bfc_status bfc_decode(int64_t n, int32_t L, int32_t b, int64_t m, const int32_t* i, const int32_t* j,
                      int32_t* keys)
{
    if (L < 0 || L > 24 || b < 1 || n != (int64_t)b << L || m < 0) return fail(nullptr, BFC_EINVAL, "bad sizes");
    if (m == 0) return BFC_OK;
    if (!i || !j || !keys) return fail(nullptr, BFC_EINVAL, "null argument");
    for (int64_t e = 0; e < m; ++e)
        if (i[e] < 0 || i[e] >= n || j[e] < 0 || j[e] >= n) return fail(nullptr, BFC_EINVAL, "index outside [0, n)");
    const int NL = L + 2;
    int32_t *di = nullptr, *dj = nullptr, *dk = nullptr;
    cudaError_t e = cudaMalloc((void**)&di, m * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dj, m * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dk, (size_t)m * NL * 4);
    if (e == cudaSuccess) e = cudaMemcpy(di, i, m * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dj, j, m * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        launch_all_keys(di, dj, m, L, b, dk, 0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(keys, dk, (size_t)m * NL * 4, cudaMemcpyDeviceToHost);
    cudaFree(di);
    cudaFree(dj);
    cudaFree(dk);
    if (e != cudaSuccess) return fail(nullptr, BFC_ECUDA, std::string("decode: ") + cudaGetErrorString(e));
    return BFC_OK;
}

bfc_status bfc_level_groups(bfc_ctx* ctx, int32_t level, int64_t* ngroups, int32_t* grouped)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    if (level < 0 || level > c->L + 1) return fail(c, BFC_EINVAL, "level outside [0, L+1]");
    const bool mid = level >= 1 && level <= c->L && (int)c->grp.size() > level;
    if (ngroups) *ngroups = mid ? c->grp[level].ngroups : 0;
    if (grouped) *grouped = level_grouped(c, level) ? 1 : 0;
    return BFC_OK;
}

bfc_status bfc_get_order(bfc_ctx* ctx, int32_t level, int32_t* perm, int32_t* seg)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    if (level < 0 || level > c->L + 1) return fail(c, BFC_EINVAL, "level outside [0, L+1]");
    const int64_t K = (level == 0 || level == c->L + 1) ? c->n : c->S;
    if (perm) BFC_CK(c, cudaMemcpyAsync(perm, c->perm[level], c->N * 4, cudaMemcpyDeviceToHost, c->stream));
    if (seg) BFC_CK(c, cudaMemcpyAsync(seg, c->seg[level], (K + 1) * 4, cudaMemcpyDeviceToHost, c->stream));
    return sync(c);
}

bfc_status bfc_profile_enable(bfc_ctx* ctx, int32_t enable)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    BFC_TRY(sync(c));
    c->prof = enable != 0;
    c->prof_rec.clear();
    return BFC_OK;
}

bfc_status bfc_profile_read(bfc_ctx* ctx, bfc_kernel_profile* out, int32_t cap, int32_t* count)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return BFC_EINVAL;
    BFC_TRY(sync(c));
    if (count) *count = (int32_t)c->prof_rec.size();
    for (int q = 0; q < cap && q < (int)c->prof_rec.size(); ++q) {
        memset(out[q].name, 0, sizeof(out[q].name));
        strncpy(out[q].name, c->prof_rec[q].name.c_str(), sizeof(out[q].name) - 1);
        out[q].launches = c->prof_rec[q].launches;
        out[q].total_ms = c->prof_rec[q].total_ms;
    }
    return BFC_OK;
}

bfc_status bfc_inject_fault(bfc_ctx* ctx, int32_t kind)
{
    if (!ctx) return fail(nullptr, BFC_EINVAL, "null context");
    Ctx* c = (Ctx*)ctx;
    if (kind < 0 || kind > 2) return fail(c, BFC_EINVAL, "fault kind must be 0, 1 or 2");
    BFC_CK(c, cudaStreamSynchronize(c->stream));
    c->inject = kind;
    drop_graph(c);   // the captured sweep holds the kernels' arguments
    return BFC_OK;
}

const char* bfc_last_error(const bfc_ctx* ctx)
{
    const Ctx* c = (const Ctx*)ctx;
    return c ? c->err.c_str() : g_create_err.c_str();
}

void bfc_destroy(bfc_ctx* ctx)
{
    Ctx* c = (Ctx*)ctx;
    if (!c) return;
    if (c->own_stream) cudaStreamSynchronize(c->own_stream);
    if (c->stream && c->stream != c->own_stream) cudaStreamSynchronize(c->stream);
    drop_graph(c);
    for (void* p : c->allocs) cudaFree(p);
    for (auto& p : c->prof_pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

}  // extern "C"
