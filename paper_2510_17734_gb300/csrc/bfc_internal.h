// Internal definitions of libbfc: the context object and host-side helpers.
// Not part of the ABI (include/bfc.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bfc.h"

namespace bfc {

// Per-kernel CUDA-event accounting (bfc_profile_enable / bfc_profile_read).
struct ProfRecord {
    std::string name;
    int64_t launches = 0;
    double total_ms = 0.0;
};
struct ProfPending {
    int rec;
    int kernels;
    cudaEvent_t a, b;
};

struct Ctx;
bfc_status fail(Ctx* ctx, bfc_status st, const std::string& msg);

// The entries of one middle level, inside every slice, in groups that share
// one environment: one row (by_col = 0, they share h_m) or one column
// (by_col = 1, they share w_m).  gstart[g] .. gstart[g+1] are the positions
// of group g in the level order, gseg[k] the first group of slice k.
struct GroupLevel {
    int by_col = 0;
    int64_t ngroups = 0;
    int32_t* gstart = nullptr;
    int32_t* gseg = nullptr;
    int64_t max_block = 0;   // most entries of a k_group_sums block (128 / r consecutive groups)
};

// Device buffers of one completion problem.  Level l = 0 is the S^1 (row)
// ordering of the training entries, l = 1..L the slice ordering of the middle
// factor S^{l+1}, l = L+1 the S^{L+2} (column) ordering.
struct Ctx {
    bfc_params P{};
    int64_t n = 0, N = 0, NT = 0, S = 0, Pn = 0;  // Pn: complex parameter count
    int L = 0, b = 0, r = 0;
    bool fp32 = false;              // compute type float (precision form) or double
    double ridge = 0.0;             // effective ridge floor factor (ridge_rel resolved)
    bool gram_tc = false;           // middle-level Gram on the tensor cores (tcgen05)
    int num_sms = 0;                // SMs of the context's device (persistent grids)
    size_t vsz = 16;                // bytes of one complex compute value
    cudaStream_t stream = nullptr, own_stream = nullptr;
    std::string err;

    // observed data, original order
    int32_t *d_i = nullptr, *d_j = nullptr;
    double2* d_t = nullptr;
    int32_t *d_it = nullptr, *d_jt = nullptr;
    double2* d_tt = nullptr;

    // orderings (built once per Omega)
    std::vector<int32_t*> seg;   // L+2 segment offset arrays
    std::vector<void*> tval;     // L+2 value arrays in level order (compute type)
    std::vector<int32_t*> nxt;   // l = 0..L : position in order l+1 of the entry at position p of order l
    std::vector<int32_t*> prv;   // l = 1..L : position in order l-1 (index 0 unused)
    int32_t* jL = nullptr;       // column index of the entries in order L
    std::vector<int32_t*> perm;  // L+2: entry index at each position of order l
    std::vector<GroupLevel> grp; // L+2: row / column groups of the middle levels (empty otherwise)
    void* grec = nullptr;        // group records [s | M | v] of the level being solved (grouped Gram)
    double grp_max_ratio = 0.0;  // a middle level's Gram runs per group when groups / entries < this
                                 // (next to the tensor-core kernel)
    double grp_cuda_ratio = 0.0; // the same next to the per-entry CUDA-core kernel

    // environments (compute type): W[l] (l = 0..L) in order l, two H buffers
    void* W = nullptr;
    void* H[2] = {nullptr, nullptr};
    void* Rres[2] = {nullptr, nullptr};  // residual carried along the orders (gradient)
    void* rec = nullptr;              // per-block normal-equation records [K packed | y]
    double2* fb = nullptr;            // FP64 refinement / fallback records (precision form)
    int32_t* fblist = nullptr;        // slices handed to the FP64 fallback in the current level

    // factors: FP64 master and compute-type copies (alias when double)
    double2 *z1d = nullptr, *Zd = nullptr, *zLd = nullptr;
    void *z1t = nullptr, *Zt = nullptr, *zLt = nullptr;

    // small device scratch: reductions and counters
    double* d_red = nullptr;          // partial sums, size red_cap
    int64_t red_cap = 0;
    double* d_scalars = nullptr;      // 16 doubles of results
    // 8 counters: [0] singular systems, [1] FP64 fallbacks and [2] refinement
    // steps of the sweep, [3] fallback list length of the current level,
    // [4] index-check flag of bfc_eval
    unsigned long long* d_count = nullptr;
    void* d_tmp = nullptr;            // growable scratch (eval inputs, etc.)
    size_t tmp_cap = 0;

    // sweep bookkeeping
    int32_t sweeps_done = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // one captured sweep (kernels and memsets only), replayed by the batch
    cudaGraphExec_t sweep_graph = nullptr;
    cudaGraph_t sweep_graph_src = nullptr;
    int64_t graph_launches = 0;     // kernels in the captured sweep
    bool graph_tc = false;          // Gram kernel the capture used

    // ADAM moments (bfc_adam), packed like the factors, allocated on first use
    double2* adam_m = nullptr;
    double2* adam_v = nullptr;

    // failure injection of the tests (bfc_inject_fault): 0 off, 1 bulk copies
    // of the solve and gradient kernels not issued (their bounded waits
    // expire), 2 the device error word set on the host before the status read
    int32_t inject = 0;

    // profiling
    bool prof = false;
    int64_t n_launch = 0;           // kernels launched by this context so far
    std::vector<ProfRecord> prof_rec;
    std::vector<ProfPending> prof_pending;
    std::vector<cudaEvent_t> ev_pool;

    std::vector<void*> allocs;        // everything cudaMalloc'ed by this context
};

// Allocation helper: records the pointer for bfc_destroy.
bfc_status dalloc(Ctx* c, void** p, size_t bytes, const char* what);
bfc_status ensure_tmp(Ctx* c, size_t bytes);

// Whether middle level m runs the grouped Gram: gram_impl 0, r = 4 or 8,
// and fewer groups than the threshold against the per-entry kernel in use.
bool level_grouped(const Ctx* c, int m);

// Profiling scope around one launch.
struct ProfScope {
    Ctx* c;
    int rec = -1;
    int kernels = 1;
    cudaEvent_t a = nullptr;
    // `kernels`: how many kernels the scope launches (added to Ctx::n_launch
    // whether or not profiling is on).
    ProfScope(Ctx* ctx, const char* name, int kernels = 1);
    ~ProfScope();
    // the scope launched k more kernels than it was opened with
    void add_kernels(int k)
    {
        kernels += k;
        c->n_launch += k;
    }
};
void prof_collect(Ctx* c);

}  // namespace bfc

#define BFC_CK(ctx, call)                                                          \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return ::bfc::fail((ctx), BFC_ECUDA,                                   \
                               std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define BFC_LAUNCH_CHECK(ctx, name)                                                 \
    do {                                                                            \
        cudaError_t e_ = cudaGetLastError();                                        \
        if (e_ != cudaSuccess)                                                      \
            return ::bfc::fail((ctx), BFC_ECUDA,                                    \
                               std::string("launch ") + (name) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define BFC_TRY(call)                        \
    do {                                     \
        bfc_status s_ = (call);              \
        if (s_ != BFC_OK) return s_;         \
    } while (0)
