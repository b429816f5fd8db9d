/*
 * bfc.h -- C ABI of the GB300 butterfly tensor completion library (libbfc.so).
 *
 * The operation: given an n x n complex matrix T observed on an index set
 * Omega, find butterfly factors S = {S^1, ..., S^{L+2}} (n = b * 2^L, leaf
 * size b, butterfly rank r) minimizing
 *     f(S) = 1/2 sum_{(i,j) in Omega} |x_ij(S) - t_ij|^2 + lambda/2 ||S||^2,
 * where x_ij(S) is the tensor-network entry formula Eq. (BF_tensor_rep),
 * Sec. 3.1, and the objective is Eq. (BF_objective), Sec. 4, with the
 * regularization of Sec. 4.1.1.  Alternating least squares follows Alg. 1.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Tree bits (Eq. (indices)): p_i = floor(i / b) is the L-bit tree prefix of
 * row i with i_0 its most significant bit; i_L = i mod b.  Same for columns.
 *
 * Factor layout after the App. A.2 reshape (Eq. (reshaped_tensors)):
 *   z1[i][a]            fiber s^1(i_0..i_L, :),           n x r
 *   Z[m][k][a][c]       slice S^{m+1}(k, :, :), m = 1..L, k < 2^{L+1},
 *                       k = psi^{-1}(i_0..i_{L-m}, j_0..j_{m-1}) MSB-first,
 *                       i.e. k = ((p_i >> (m-1)) << m) | (p_j >> (L-m));
 *                       a is the left rank index r_m, c the right one r_{m+1}
 *   zL[j][c]            fiber s^{L+2}(j_0..j_L, :),       n x r
 *   x_ij = z1[i]^T Z[1][k_2] ... Z[L][k_{L+1}] zL[j]   (no conjugation).
 *
 * "Packed" factor vectors are complex128, interleaved (re, im), of
 * bfc_num_params() complex numbers: [ z1 : n r ][ Z : L 2^{L+1} r^2 ][ zL : n r ].
 *
 * Complex values (t, outputs) are always interleaved complex128 (2 doubles).
 * Index arrays are int32.
 *
 * Ownership: the caller owns every array it passes; bfc_create copies the
 * observed data to the device, so inputs may be freed after it returns.
 * Output arrays are caller-allocated.  The context owns all device memory and
 * releases it in bfc_destroy.  Pointers are host pointers unless
 * params.values_on_device is 1, in which case the data arrays passed to
 * bfc_create / bfc_set_factors / bfc_get_factors / bfc_eval / bfc_grad must
 * be device pointers (for example from torch tensors).
 *
 * Errors: every call returns a bfc_status; no C++ exception crosses the ABI.
 * bfc_last_error() gives a message for the last failing call on a context.
 * Calls on one context are ordered on its stream (bfc_set_stream) and return
 * after the stream work they issued has finished.  Use one context per host
 * thread.
 */
#ifndef BFC_H
#define BFC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bfc_ctx bfc_ctx;

typedef enum {
    BFC_OK = 0,
    BFC_EINVAL = 1,      /* invalid argument: sizes, indices, duplicates, NaN/Inf */
    BFC_ENOMEM = 2,      /* device or host allocation failed */
    BFC_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    BFC_ESINGULAR = 4,   /* reserved: a solve could not proceed at all */
    BFC_ETIMEOUT = 5,    /* a bounded device-side wait gave up */
    BFC_ENONFINITE = 6   /* a result became NaN or Inf */
} bfc_status;

typedef enum {
    /* Everything in FP64: environment chains, normal-equation sums, solves. */
    BFC_PREC_FP64 = 0,
    /* Precision form: chains and normal-equation sums in complex64 with
     * compensated accumulation (tensor cores for r <= 8, see gram_impl);
     * per-slice solves refined to FP64-level accuracy (complex64 Cholesky,
     * iterative refinement with a double-float residual and solution, FP64
     * Cholesky fallback); factor master copy in FP64. */
    BFC_PREC_C64_FP64SOLVE = 1
} bfc_precision;

typedef struct {
    int64_t n;              /* matrix size; must equal b * 2^L               */
    int32_t L;              /* butterfly levels, 0 <= L <= 24 (L = 0: low-rank) */
    int32_t b;              /* leaf size (the paper's c), >= 1               */
    int32_t r;              /* butterfly rank, 1 <= r <= 12                  */
    double lambda;          /* regularization added to every system, >= 0    */
    int32_t prec;           /* bfc_precision                                 */
    int32_t max_sweeps;     /* bfc_complete: sweep limit                     */
    double tol;             /* bfc_complete: stop when train rel. err < tol  */
    uint64_t seed;          /* bfc_complete with init_kind 1: random start   */
    int32_t init_kind;      /* bfc_complete: 0 = current factors,
                               1 = low-rank completion (Alg. 1 with L = 0,
                                   rank lr_rank, lr_sweeps sweeps) embedded
                                   exactly into the butterfly,
                               2 = the same completion converted by the
                                   randomized Alg. 2 (bfc_lowrank_to_butterfly)
                                   with CN(0, 1) Gaussians from SplitMix64
                                   (seed + 1)                              */
    int32_t lr_rank;        /* rank R of the low-rank start (<= r)           */
    int32_t lr_sweeps;      /* sweeps of low-rank completion                 */
    int32_t values_on_device; /* 1: data pointers are device pointers        */
    int32_t refine_sweeps;  /* precision form: FP64 sweeps appended by
                               bfc_complete after the complex64 sweeps       */
    double ridge_rel;       /* ridge floor: every system is solved with
                               max(lambda, ridge_rel * trace(K) / dim).
                               0 selects the default (2^-20, the complex64
                               rounding level of the normal equations, in the
                               precision form; none in FP64); < 0 disables  */
    int32_t gram_impl;      /* per-slice normal equations of the middle
                               levels.  0 = automatic: for r = 4 or 8, a
                               level whose row (or column) groups are few
                               against its entries (below group_ratio of
                               them) runs the grouped Gram (the entries of one row
                               / column of a slice share an environment, so
                               the sums are taken per group and the Gram is
                               the sum of Kronecker products of the group
                               sums; both precisions); the other levels run
                               the per-entry kernel of 2 (precision form,
                               r <= 8) or of 1.  1 = per-entry CUDA cores
                               (complex64 FMA, or FP64) at every level.  2 =
                               per-entry tensor cores (tcgen05, three-term
                               TF32 products, Kahan-folded every 32 entries)
                               at every level in the precision form for
                               r <= 8, CUDA cores otherwise.  Any other
                               value is BFC_EINVAL.                         */
    int32_t lr2bf_oversample; /* oversampling p of Alg. 2 for init_kind 2
                               (0 selects 5); r + p <= 32                   */
    double group_ratio;     /* gram_impl 0: groups-per-entry threshold of the
                               grouped Gram.  0 selects the default (0.1
                               next to the tensor-core kernel, 0.9 next to
                               the CUDA-core one); < 0 never groups; > 0
                               is used as given                             */
} bfc_params;

typedef struct {
    int32_t sweep;          /* 1-based sweep number                          */
    double train_rel_err;   /* Eq. (BF_convergence) on the training set      */
    double test_rel_err;    /* same on the test set (-1 if none)             */
    double objective;       /* f(S) after the sweep                          */
    double sweep_ms;        /* device time of the sweep (CUDA events)        */
    double entries_per_s;   /* training entries / sweep time                 */
    int64_t singular_slices;/* systems left unchanged (Cholesky breakdown)   */
    int64_t refined_fallbacks; /* precision form: FP64 Cholesky fallbacks    */
    int64_t refine_steps;   /* precision form: refinement steps taken        */
    int64_t launches;       /* kernels this call launched (sweep + errors)   */
    int32_t gram_impl;      /* per-entry middle-level Gram kernel of the
                               precision form (levels not on the grouped
                               Gram): 0 tensor cores, 1 CUDA cores; -1 FP64
                               path                                         */
    int32_t batch_launches; /* bfc_batch_complete: graph launches that ran
                               the sweeps after the autotuning (1: all of
                               them in one launch); 0 elsewhere             */
} bfc_sweep_stats;

typedef struct {
    char name[48];          /* kernel name                                   */
    int64_t launches;       /* launches since profiling was enabled          */
    double total_ms;        /* summed CUDA-event durations                   */
} bfc_kernel_profile;

/* Number of complex parameters 2 n r + L 2^{L+1} r^2 (Sec. 2.2 memory count
 * with the App. A.2 reshape).  Returns -1 for invalid sizes. */
int64_t bfc_num_params(int64_t n, int32_t L, int32_t b, int32_t r);

/* Create a context for one completion problem (Sec. 4 problem statement:
 * T on Omega, sizes, rank, lambda).  Copies the nnz training entries
 * (i[e], j[e], t[e]) and ntest test entries (it, jt, tt; ntest may be 0) to
 * the device, validates them (indices in [0, n), no duplicate (i, j) in the
 * training set since Omega is a set, finite values), builds the per-factor
 * entry orderings (the "transpose the sparse tensor according to the index
 * being solved for" step of App. A.2) and zero-initializes the factors.
 * On success *out receives the context; on failure *out is NULL.
 * Errors: EINVAL (n != b 2^L, r out of range, lambda < 0, nnz <= 0,
 * bad index, duplicate, NaN/Inf), ENOMEM, ECUDA. */
bfc_status bfc_create(const bfc_params* params, int64_t nnz, const int32_t* i,
                      const int32_t* j, const double* t, int64_t ntest,
                      const int32_t* it, const int32_t* jt, const double* tt,
                      bfc_ctx** out);

/* Run all further work of this context on `cuda_stream` (a cudaStream_t;
 * NULL selects the context's own stream). */
bfc_status bfc_set_stream(bfc_ctx* ctx, void* cuda_stream);

/* Replace the factors by a packed complex128 vector (layout above). */
bfc_status bfc_set_factors(bfc_ctx* ctx, const double* packed);

/* Copy the current factors (FP64 master copy) into a packed vector. */
bfc_status bfc_get_factors(bfc_ctx* ctx, double* packed);

/* Evaluate x_ij (Eq. (BF_tensor_rep)) for m index pairs; out receives m
 * interleaved complex128 values.  Arithmetic follows the context precision
 * (FP64, or complex64 chains in the precision form).  EINVAL on an index
 * outside [0, n). */
bfc_status bfc_eval(bfc_ctx* ctx, int64_t m, const int32_t* i, const int32_t* j,
                    double* out);

/* One ALS sweep (Alg. 1): S^1 fibers, then S^2 .. S^{L+1} slices in order,
 * then S^{L+2} fibers, each block the exact minimizer of f with the newest
 * values of all other factors (complex normal equations
 * K = sum conj(a) a^T + lambda I, y = sum conj(a) t).  A system whose
 * Cholesky pivot falls to <= 0 (<= 1e-14 trace(K) when lambda = 0) keeps its
 * old values and is counted in singular_slices.  `out` may be NULL.
 * Unless kernel profiling is on, the first call captures the sweep's kernels
 * into a CUDA graph on the context stream and every call launches that graph
 * (same kernels, same order); a stream that cannot be captured runs them
 * directly.  BFC_ETIMEOUT if a bounded device wait (the tensor-core Gram's
 * mbarriers, the bulk copies of the solve) expired; the sweep's results are
 * then undefined and the context stays usable. */
bfc_status bfc_als_sweep(bfc_ctx* ctx, bfc_sweep_stats* out);

/* Gradient of f with respect to all parameters (Eqs. (grad_butterfly_1),
 * (grad_butterfly_l), (grad_butterfly_last) with z = x - t), packed as
 * df/dRe + i df/dIm; the regularization term lambda S is added when
 * include_reg is nonzero.  grad_packed (may be NULL) receives the packed
 * gradient, *objective (may be NULL) the value of f (with or without the
 * regularization term, matching include_reg).  BFC_ETIMEOUT if a bounded
 * device wait (the bulk copies of the middle levels) expired; the gradient
 * is then undefined and the context stays usable. */
bfc_status bfc_grad(bfc_ctx* ctx, int32_t include_reg, double* grad_packed,
                    double* objective);

/* Gradient completion: `iters` iterations of limited-memory BFGS on the 2P
 * real parameters (the packed factors viewed as doubles) of the regularized
 * objective f, with the gradients of bfc_grad (Eqs. (grad_butterfly_*)).
 * Two-loop recursion with `memory` pairs (1..64) and H0 = gamma I (gamma =
 * s^T y / y^T y of the newest pair); backtracking Armijo line search
 * (c1 = 1e-4, step halved, at most 30 trials) starting from step 1, or from
 * 1 / ||g|| before the first pair; a pair is kept only if
 * s^T y > 1e-12 ||s|| ||y||.  The factors end at the last accepted point.
 * history (may be NULL) receives per-iteration training / test errors and f;
 * *done (may be NULL) the iterations run. */
bfc_status bfc_lbfgs(bfc_ctx* ctx, int32_t iters, int32_t memory, bfc_sweep_stats* history,
                     int32_t history_cap, int32_t* done);

/* ADAM completion (Alg. 4 with the update of Alg. 3, Sec. 4.1.2): `iters`
 * outer iterations t = 1 .. iters.  Each updates S^1, S^2 .. S^{L+1},
 * S^{L+2} in turn, every factor with the gradient of f (Eqs.
 * (grad_butterfly_1/_l/_last), the regularization term lambda s included)
 * taken at the newest values of all other factors, then
 *   m <- beta1 m + (1 - beta1) g,  v <- beta2 v + (1 - beta2) g^2,
 *   s <- s - alpha (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + sigma)
 * on the real and the imaginary part of every complex parameter separately
 * (FP64 moments and master factors; the residuals and gradient sums follow
 * the context precision).  The moments start at zero on every call.  Stops
 * after the iteration whose training error (Eq. (BF_convergence)) is below
 * params.tol.  history (may be NULL) receives up to history_cap iteration
 * records, *done (may be NULL) the iterations run.  EINVAL for iters < 0,
 * alpha <= 0, beta1 or beta2 outside [0, 1), or sigma < 0. */
bfc_status bfc_adam(bfc_ctx* ctx, int32_t iters, double alpha, double beta1, double beta2, double sigma,
                    bfc_sweep_stats* history, int32_t history_cap, int32_t* done);

/* ADF completion (Alg. 5, Sec. 4.1.3, with the orthogonalization sweeps of
 * App. A.3): every iteration first makes every factor but S^1
 * right-orthonormal (the right-to-left sweep: LQ of the slice pairs that
 * differ in their lowest column bit, QR of the leaf blocks of S^{L+2}), forms
 * the residual G = t - x, then for S^1, S^2 .. S^{L+1}, S^{L+2} in turn moves
 * every fiber / slice s along N_s = sum_{e in s} G_e conj(a_e) - lambda s by
 * the exact minimizer of f on that line,
 *   alpha_s = ||N_s||^2 / (sum_{e in s} |a_e . N_s|^2 + lambda ||N_s||^2),
 * updates G, and (except for S^{L+2}) QR-factors the factor's bond groups
 * (R with a real positive diagonal) and multiplies R into the next factor.
 * Stopping, history and done as bfc_adam.  EINVAL when b < r (the leaf
 * blocks must have full column rank) or iters < 0. */
bfc_status bfc_adf(bfc_ctx* ctx, int32_t iters, bfc_sweep_stats* history, int32_t history_cap, int32_t* done);

/* Butterfly matrix-vector product (Eq. (butterfly-mat-vec), Sec. 3.2):
 * U = X(S) V for nvec vectors in O((n r + L 2^{L+1} r^2) nvec) work, by the
 * level-by-level contraction of the factors: the leaf sums of S^{L+2} with
 * the vectors, then S^{L+1} .. S^2 each summing out one column bit, then
 * S^1.  V and U are n x nvec row-major complex128 (V[j * nvec + q]), host or
 * device arrays per params.values_on_device; arithmetic in the context
 * precision.  EINVAL unless 1 <= nvec <= 4096. */
bfc_status bfc_matvec(bfc_ctx* ctx, int32_t nvec, const double* V, double* U);

/* Low-rank start (Sec. 4.2): low-rank matrix completion of rank R <= r from
 * the caller's starting factors A0, B0 (n x R packed complex128, X = A B^T),
 * `sweeps` sweeps of Alg. 1 with L = 0 on the GPU, then the exact embedding
 * z1 = A, every middle slice = identity, zL = B (columns R..r-1 zero).
 * Sets the context's factors.  A0/B0 follow values_on_device. */
bfc_status bfc_lowrank_init(bfc_ctx* ctx, int32_t R, int32_t sweeps,
                            const double* A0, const double* B0);

/* Randomized low-rank to butterfly conversion (Alg. 2, Sec. 4.2): sets the
 * factors to a butterfly of X = A B^T (A, B: n x R complex128, 1 <= R <= r;
 * host or device per params.values_on_device), in FP64.
 *  1. M = A (B^T O_0), N = B (A^T O_0); for every leaf block, QR with column
 *     pivoting of its b rows of M (of N) gives the block's rows of S^1
 *     (S^{L+2}): the first r columns of Q; V = Q^H A(block) (W = Q^H B(block))
 *     are its coefficients.
 *  2. For the left levels l = 1 .. H = floor(L / 2): per column block nu the
 *     sketch B(nu)^T O_l; the two slices of S^{l+1} that differ in i_{L-l}
 *     are the halves of Q of the QRCP of [V_0; V_1] B(nu)^T O_l (their two
 *     coefficient blocks stacked), and V := Q^H [V_0; V_1].  The right levels
 *     l = 1 .. L - H fill S^{L+2-l} in the mirror order (pairs differing in
 *     j_{L-l}, sketch A(tau)^T O'_l, halves of Q transposed).
 *  3. The slices of S^{H+1} (z1 when H = 0) are right-multiplied by V W^T.
 * `gaussians` holds the CN(0, 1) sketch matrices, r + p columns each,
 * row-major, packed O_0 (n rows), O_1 .. O_H and O'_1 .. O'_{L-H}
 * (b 2^{L-l} rows each); same memory kind as A and B.  With R <= r the
 * butterfly reproduces A B^T to rounding; a leaf block smaller than r
 * (b < r) gets b columns of Q and zeros (its b rows are spanned exactly).
 * EINVAL unless 1 <= R <= r, p >= 0 and r + p <= 32. */
bfc_status bfc_lowrank_to_butterfly(bfc_ctx* ctx, int32_t R, const double* A, const double* B, int32_t p,
                                    const double* gaussians);

/* Full workflow (Sec. 4.3): optional low-rank start (init_kind 1, with a
 * CN(0, sigma^2) SplitMix64 start from params.seed), then ALS sweeps until
 * the training error (Eq. (BF_convergence)) is below params.tol or
 * params.max_sweeps sweeps ran, then params.refine_sweeps FP64 sweeps in the
 * precision form.  history (may be NULL) receives up to history_cap sweep
 * records; *nsweeps (may be NULL) the number of sweeps run. */
bfc_status bfc_complete(bfc_ctx* ctx, bfc_sweep_stats* history, int32_t history_cap,
                        int32_t* nsweeps);

/* Batched form: the full workflow of bfc_complete (start, sweeps until
 * params.tol or params.max_sweeps, FP64 refinement sweeps) for `count`
 * independent problems, each with its own context and params.  Each
 * problem's sweep is captured once as a CUDA graph; every round launches
 * one graph whose child graphs are the sweeps of all unfinished problems
 * (rebuilt only when that set changes), so the problems run concurrently
 * on the GPU from a single launch per round.  In the precision form with
 * gram_impl 0, the per-entry Gram kernel is autotuned per rank: the first
 * problem of each rank r <= 8 runs one warm-up and one timed sweep with each kernel
 * (ordinary sweeps, counted) and the faster serves all problems of that
 * rank.  last (may be NULL) receives the last sweep's statistics of each
 * problem.  A context may appear once; contexts must live on the current
 * device.  No counterpart in the paper's listings: the batch is the
 * independent-problem parallelism of Sec. 4 applied across problems. */
bfc_status bfc_batch_complete(int32_t count, bfc_ctx* const* ctxs, bfc_sweep_stats* last);

/* Gauge fixing (left orthogonalization).  Eq. (BF_tensor_rep) is unchanged
 * when an invertible r x r matrix is inserted on a bond between two factors
 * (the network's gauge freedom).  Level by level from S^1, every bond group
 * is factored M = Q R, with R upper triangular with a real positive
 * diagonal (unique), and replaced by Q; R moves into the next factor.  The
 * groups are: the b x r leaf blocks of z1; then, for each middle level and
 * bond, the two slices sharing it, stacked 2r x r.  Every factor but zL
 * ends left-orthonormal; zL carries the norm.  The FP64 factors are
 * updated in place (entries are unchanged to rounding).  Needs b >= r.
 * The paper has no counterpart: used to give the learned start consistent
 * training targets. */
bfc_status bfc_canonicalize(bfc_ctx* ctx);

/* ---- Learned initializer (a small MLP from problem parameters to factors) */

/* Opaque model: in -> hidden -> hidden -> out with GELU after both hidden
 * layers and a linear output; FP32 master weights with Adam state, BF16
 * weights in every forward / backward kernel, FP32 activations and
 * accumulation.  Inputs are mapped to [-1, 1] by stored ranges; the network
 * predicts per-output standardized values (stored mean and standard
 * deviation).  The model owns its device memory; one model per host thread.
 * The paper has no counterpart: this is the learned replacement of the
 * low-rank start of Sec. 4.2. */
typedef struct bfc_mlp bfc_mlp;

/* He-normal weights from SplitMix64(seed), zero biases, identity scaling.
 * 1 <= in_dim <= 64, 1 <= hidden <= 256, 1 <= out_dim <= 2^31. */
bfc_status bfc_mlp_create(int32_t in_dim, int32_t hidden, int64_t out_dim, uint64_t seed, bfc_mlp** out);

/* Sizes (any pointer may be NULL); parameter count of the flat layout
 * [W1 (in x hidden) | b1 | W2 (hidden x hidden) | b2 | W3 (hidden x out) |
 * b3], each W input-major (W[k][n] at k * fan_out + n). */
void bfc_mlp_dims(const bfc_mlp* m, int32_t* in_dim, int32_t* hidden, int64_t* out_dim);
int64_t bfc_mlp_num_params(const bfc_mlp* m);

/* Flat FP32 master parameters as host doubles (get) or from host doubles
 * (set; the BF16 copy is refreshed). */
bfc_status bfc_mlp_get_params(bfc_mlp* m, double* params);
bfc_status bfc_mlp_set_params(bfc_mlp* m, const double* params);

/* Input ranges [lo, hi] (in_dim each, hi > lo) and output mean / standard
 * deviation (out_dim each, std > 0), host arrays. */
bfc_status bfc_mlp_set_scaling(bfc_mlp* m, const double* in_lo, const double* in_hi,
                               const double* out_mean, const double* out_std);

/* Predictions y[s * out_dim + q] (de-standardized) for `count` host inputs
 * x[s * in_dim + q]. */
bfc_status bfc_mlp_forward(bfc_mlp* m, int32_t count, const double* x, double* y);

/* Mean squared error of the standardized prediction against the
 * standardized targets of 1 <= count <= 32 samples, and its gradient with
 * respect to the flat parameters (grads may be NULL; loss may be NULL). */
bfc_status bfc_mlp_grad(bfc_mlp* m, int32_t count, const double* x, const double* y,
                        double* grads, double* loss);

/* Training on `count` samples: sets the input ranges and output scaling from
 * the data, then `epochs` passes of Adam (lr, beta 0.9 / 0.999) over shuffled
 * mini-batches of `batch` (1..32) samples (SplitMix64(seed) order).
 * loss_history (may be NULL) receives the mean batch loss of each epoch. */
bfc_status bfc_mlp_train(bfc_mlp* m, int32_t count, const double* x, const double* y, int32_t epochs,
                         int32_t batch, double lr, uint64_t seed, double* loss_history);

void bfc_mlp_destroy(bfc_mlp* m);

/* Learned start: the model's prediction for the inputs (omega / (pi n),
 * offset) becomes the context's factors (model output size must be 2 P).
 * With allow_fallback, the low-rank start of bfc_complete's init_kind 1 is
 * also computed and whichever has the lower training error (Eq.
 * (BF_convergence)) is kept.  *used_learned (may be NULL) tells which;
 * *start_err (may be NULL) receives the kept start's training error. */
bfc_status bfc_init_learned(bfc_ctx* ctx, bfc_mlp* model, double omega, double offset,
                            int32_t allow_fallback, int32_t* used_learned, double* start_err);

/* Measured FP32 and FP64 FMA throughput of the current device in TFLOP/s
 * (dependent-FMA chains, all SMs, best of five launches; about one second).
 * The denominators of the CUDA-core kernels' ALU rooflines.  No counterpart
 * in the paper. */
bfc_status bfc_measure_alu_peaks(double* fp32_tflops, double* fp64_tflops);

/* Index decoding on the GPU (Eq. (indices) and the App. A.2 slice ids):
 * for m host pairs (i[e], j[e]) writes keys[e * (L+2) + l] = i for l = 0, the
 * slice id k_{l+1} of S^{l+1} for l = 1..L, and j for l = L+1.  These are
 * the keys by which bfc_create orders the entries.  Host arrays; EINVAL on
 * bad sizes or an index outside [0, n). */
bfc_status bfc_decode(int64_t n, int32_t L, int32_t b, int64_t m, const int32_t* i,
                      const int32_t* j, int32_t* keys);

/* The entry ordering of one factor level (0 = S^1 rows, 1..L = slices of
 * S^{l+1}, L+1 = S^{L+2} columns): perm[p] is the training entry (index into
 * the arrays given to bfc_create) at position p, stable in input order within
 * a key; seg[k] .. seg[k+1] is the range of key k (n + 1 values for levels 0
 * and L+1, 2^{L+1} + 1 otherwise).  Host arrays; either may be NULL. */
bfc_status bfc_get_order(bfc_ctx* ctx, int32_t level, int32_t* perm, int32_t* seg);

/* Row / column groups of one middle level (1..L): inside every slice of
 * S^{level+1}, the entries of one row (levels with 2 level <= L + 1) or of
 * one column share the environment on that side; *ngroups receives the
 * number of such groups over all slices (0 where groups are not formed: the
 * outer levels 0 and L+1, or a level whose composite sort key would not fit
 * 32 bits), *grouped whether this context's sweeps run the level's normal
 * equations per group (gram_impl, group_ratio).  Either pointer may be NULL;
 * EINVAL on a level outside [0, L+1].  No counterpart in the paper: the
 * grouping is an implementation of the slice sums of Alg. 1. */
bfc_status bfc_level_groups(bfc_ctx* ctx, int32_t level, int64_t* ngroups, int32_t* grouped);

/* Per-kernel device-time accounting with CUDA events on the context stream
 * (off by default).  Enabling resets the counters. */
bfc_status bfc_profile_enable(bfc_ctx* ctx, int32_t enable);
/* Copy up to cap records; *count receives the number of distinct kernels. */
bfc_status bfc_profile_read(bfc_ctx* ctx, bfc_kernel_profile* out, int32_t cap,
                            int32_t* count);

/* Allocation-free residual sums.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- code embedded in a
 * host application whose allocator or memory pool owns all device memory and
 * forbids other allocations, and latency-sensitive callers that cannot
 * accept an allocation (which may synchronize the device or fail) at call
 * time.  It allocates nothing: no context, no cudaMalloc or cudaFree, no
 * allocating library routine.
 *
 * Computes, for the butterfly with packed complex128 factors `factors` (the
 * layout above, sizes n = b 2^L and rank r in [1, 10]), over m entries the
 * squared residual norm and the squared data norm:
 *     sums[0] = sum_e |t_e - x_{i_e j_e}|^2,   sums[1] = sum_e |t_e|^2,
 * with FP64 entry evaluation.  All of factors, i, j, t (m interleaved
 * complex128) and sums (2 doubles) are DEVICE pointers owned by the caller:
 * device (or managed) memory usable on the current device, with factors and
 * t 16-byte aligned (they are read as 16-byte vectors), i and j 4-byte and
 * sums 8-byte aligned.  The work is enqueued on `stream` (a cudaStream_t,
 * NULL = default stream) and the call returns without waiting; sums is
 * valid once the stream reaches this point.
 * Scratch: per-block partial sums live in one fixed file-scope device array
 * of the library (256 KiB, held by every GPU that loads the library until the
 * process exits), so m may be at most 4,194,304; larger m, bad sizes, NULL,
 * misaligned or host pointers return BFC_EINVAL (message in
 * bfc_last_error(NULL)) without launching anything.  m = 0 sets both sums
 * to 0.  An index outside [0, n) makes both sums NaN.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current and keeps it; make that
 * first call before any stream capture, and do not use the library across a
 * cudaDeviceReset.  Every call shares the array and leaves its partials in it
 * (the bad-index flag is cleared at the start of each call): calls that
 * overlap on the GPU, on any streams, race and give wrong sums. */
bfc_status bfc_residual_noalloc(int64_t n, int32_t L, int32_t b, int32_t r,
                                const double* factors, int64_t m, const int32_t* i,
                                const int32_t* j, const double* t, double* sums,
                                void* stream);

/* Failure injection for tests of the error paths; the paper has no
 * counterpart.  Nothing faults on the GPU: kind 1 makes the kernels of this
 * context skip issuing the bulk copies of the middle-level solve and
 * gradient (the precision form at even rank) while still waiting for them,
 * with a wait limit of a few tries; the waits expire, the kernels load that
 * data by plain loads instead, and bfc_als_sweep / bfc_grad return
 * BFC_ETIMEOUT.  Kind 2 raises the context's device error word from the host
 * before the status read, with the same result on any path.  Kind 0 turns
 * injection off.  The setting stays until changed; the context stays usable
 * and its results are valid again once injection is off.  EINVAL for another
 * kind. */
bfc_status bfc_inject_fault(bfc_ctx* ctx, int32_t kind);

/* Message for the last failed call on ctx (or of the last failed
 * bfc_create when ctx is NULL).  Never NULL. */
const char* bfc_last_error(const bfc_ctx* ctx);

/* Release the context and all its device memory.  NULL is ignored. */
void bfc_destroy(bfc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* BFC_H */
