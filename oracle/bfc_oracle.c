/*
 * bfc_oracle.c -- plain, slow, complex128 CPU oracle for butterfly tensor
 * completion (Singh, Solomonik, Li, Liu, "Efficient Tensor Completion
 * Algorithms for Highly Oscillatory Operators", arXiv 2510.17734).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * helper with the CUDA library; the two only see the same seeded inputs.
 *
 * Everything is complex128 (C99 `double complex`), with sums taken in the
 * natural order of the entries (stable by slice, then by draw order).  The
 * loops over independent systems and entries may run on several threads
 * (bfo_set_threads); every sum is still taken by one thread in that order, so
 * the results do not depend on the thread count.
 *
 * Notation (Sec. 3.1, App. A.2):
 *   n = b * 2^L, leaf size b (the paper's c), rank r.
 *   Row index i -> tuple (i_0 .. i_{L-1}, i_L) by Eq. (indices).
 *   Middle factor S^{m+1} (m = 1..L) is stored, after the App. A.2 reshape,
 *   as 2^{L+1} slices Z^{m+1}(k, :, :) of size r x r, with slice id
 *   k_{m+1} = psi^{-1}(i_0 .. i_{L-m}, j_0 .. j_{m-1}).
 *   Outer factors: z^1(i, :) = s^1(i_0..i_L, :), z^{L+2}(j, :) likewise.
 *
 * Packed parameter vector (complex128, interleaved re/im):
 *   [ z1 : n*r ][ Z : L * 2^{L+1} * r * r ][ zL : n*r ]
 *   z1[i*r + a], Z[((m-1)*2^{L+1} + k)*r*r + a*r + c], zL[j*r + c].
 *
 * Readings of the paper used here (each also listed in the design notes):
 *  - one sweep updates S^1, then S^2 .. S^{L+1} in increasing order, then
 *    S^{L+2}, each update using the newest values of all other factors
 *    (the loop bounds of Alg. 1 are off by one as printed);
 *  - complex least squares: normal matrix K = sum conj(a) a^T + lambda I,
 *    right-hand side y = sum conj(a) t (Alg. 1 prints the real form);
 *  - Kronecker design vector a[p*r + q] = h[p] * w[q] with h the left and w
 *    the right environment, solution reshaped row-major into Z(k, p, q);
 *  - lambda I is added to every fiber / slice system ("a regularization
 *    parameter", Sec. 4.1.1);
 *  - a system whose Cholesky pivot falls below the threshold (0 when
 *    lambda > 0, 1e-14 * trace(K) when lambda == 0) keeps its old values and
 *    is counted as singular.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define BFO_MAX_L 30
#define BFO_MAX_R 64

/* Threads of the parallel loops (1 = serial).  Only loops whose iterations
 * are independent systems or entries are parallel, and every sum is taken
 * by one thread in the serial order, so any thread count gives results
 * identical bit for bit to the serial ones. */
static int g_threads = 1;

void bfo_set_threads(int threads) { g_threads = threads < 1 ? 1 : threads; }

int bfo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- indices */

/* Eq. (indices), Sec. 3.1: i_l = floor(i / (b 2^{L-l-1})) mod 2 for l < L,
 * i_L = i mod b.  Writes L+1 integers. */
void bfo_tree_bits(int64_t i, int L, int b, int32_t* bits)
{
    for (int l = 0; l < L; ++l) {
        int64_t denom = (int64_t)b;
        for (int q = 0; q < L - l - 1; ++q) denom *= 2;
        bits[l] = (int32_t)((i / denom) % 2);
    }
    bits[L] = (int32_t)(i % b);
}

/* psi^{-1}(b_0 .. b_{p-1}) = sum_q b_q 2^{p-1-q}  (App. A.2). */
int64_t bfo_psi_inv(const int32_t* bits, int p)
{
    int64_t k = 0;
    for (int q = 0; q < p; ++q) {
        int64_t w = 1;
        for (int s = 0; s < p - 1 - q; ++s) w *= 2;
        k += (int64_t)bits[q] * w;
    }
    return k;
}

/* Slice id k_{m+1} = psi^{-1}(i_0 .. i_{L-m}, j_0 .. j_{m-1}) of entry (i, j)
 * for the middle factor S^{m+1}, m = 1..L (Eq. (reshaped_tensors)). */
int64_t bfo_slice_id(int64_t i, int64_t j, int m, int L, int b)
{
    int32_t ib[BFO_MAX_L + 1], jb[BFO_MAX_L + 1], tup[2 * BFO_MAX_L + 2];
    bfo_tree_bits(i, L, b, ib);
    bfo_tree_bits(j, L, b, jb);
    int p = 0;
    for (int q = 0; q <= L - m; ++q) tup[p++] = ib[q];
    for (int q = 0; q < m; ++q) tup[p++] = jb[q];
    return bfo_psi_inv(tup, p);
}

/* Closed-form parameter count, Sec. 2.2 memory estimate with the App. A.2
 * reshape: 2 n r + L 2^{L+1} r^2 complex numbers. */
int64_t bfo_num_params(int64_t n, int L, int b, int r)
{
    (void)b;
    int64_t slices = (int64_t)1 << (L + 1);
    return 2 * n * r + (int64_t)L * slices * r * r;
}

/* ---------------------------------------------------------------- layout */

typedef struct {
    int64_t n;
    int L, b, r;
    int64_t S;         /* slices per middle factor: 2^{L+1} */
    cplx* z1;          /* n x r */
    cplx* Z;           /* L x S x r x r */
    cplx* zL;          /* n x r */
} bfo_factors;

static bfo_factors view(int64_t n, int L, int b, int r, double* packed)
{
    bfo_factors F;
    F.n = n; F.L = L; F.b = b; F.r = r;
    F.S = (int64_t)1 << (L + 1);
    F.z1 = (cplx*)packed;
    F.Z = F.z1 + n * r;
    F.zL = F.Z + (int64_t)L * F.S * r * r;
    return F;
}

static cplx* slice_ptr(const bfo_factors* F, int m, int64_t k)
{
    return F->Z + (((int64_t)(m - 1) * F->S + k) * F->r * F->r);
}

/* ------------------------------------------------------------------ eval */

/* Eq. (BF_tensor_rep): x_ij = z1(i,:)^T Z^2(k_2) ... Z^{L+1}(k_{L+1}) zL(j,:),
 * multiplied left to right, no conjugation. */
static cplx eval_entry(const bfo_factors* F, int64_t i, int64_t j)
{
    const int r = F->r;
    cplx h[BFO_MAX_R], nh[BFO_MAX_R];
    for (int a = 0; a < r; ++a) h[a] = F->z1[i * r + a];
    for (int m = 1; m <= F->L; ++m) {
        const cplx* Zk = slice_ptr(F, m, bfo_slice_id(i, j, m, F->L, F->b));
        for (int c = 0; c < r; ++c) {
            cplx s = 0;
            for (int a = 0; a < r; ++a) s += h[a] * Zk[a * r + c];
            nh[c] = s;
        }
        for (int c = 0; c < r; ++c) h[c] = nh[c];
    }
    cplx x = 0;
    for (int c = 0; c < r; ++c) x += h[c] * F->zL[j * r + c];
    return x;
}

void bfo_eval(int64_t n, int L, int b, int r, const double* packed, int64_t m,
              const int32_t* ii, const int32_t* jj, double* out)
{
    bfo_factors F = view(n, L, b, r, (double*)packed);
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (int64_t e = 0; e < m; ++e) {
        cplx x = eval_entry(&F, ii[e], jj[e]);
        out[2 * e] = creal(x);
        out[2 * e + 1] = cimag(x);
    }
}

/* x_e for every entry (in parallel), for the serial sums below. */
static cplx* eval_all(const bfo_factors* F, int64_t m, const int32_t* ii, const int32_t* jj)
{
    cplx* x = (cplx*)malloc((size_t)(m > 0 ? m : 1) * sizeof(cplx));
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (int64_t e = 0; e < m; ++e) x[e] = eval_entry(F, ii[e], jj[e]);
    return x;
}

/* Eq. (BF_convergence): ||P_Omega(T - X)||_F / ||P_Omega(T)||_F. */
double bfo_rel_err(int64_t n, int L, int b, int r, const double* packed,
                   int64_t nnz, const int32_t* ii, const int32_t* jj,
                   const double* t)
{
    bfo_factors F = view(n, L, b, r, (double*)packed);
    cplx* x = eval_all(&F, nnz, ii, jj);
    double num = 0.0, den = 0.0;
    for (int64_t e = 0; e < nnz; ++e) {
        cplx te = t[2 * e] + I * t[2 * e + 1];
        cplx d = te - x[e];
        num += creal(d * conj(d));
        den += creal(te * conj(te));
    }
    free(x);
    return den > 0.0 ? sqrt(num / den) : sqrt(num);
}

/* Regularized objective f = 1/2 sum_Omega |x - t|^2 + lambda/2 ||S||^2
 * (Eq. (BF_objective) plus the regularization of Sec. 4.1.1). */
double bfo_objective(int64_t n, int L, int b, int r, double lambda,
                     const double* packed, int64_t nnz, const int32_t* ii,
                     const int32_t* jj, const double* t)
{
    bfo_factors F = view(n, L, b, r, (double*)packed);
    cplx* x = eval_all(&F, nnz, ii, jj);
    double fit = 0.0;
    for (int64_t e = 0; e < nnz; ++e) {
        cplx te = t[2 * e] + I * t[2 * e + 1];
        cplx d = x[e] - te;
        fit += creal(d * conj(d));
    }
    free(x);
    double reg = 0.0;
    int64_t P = bfo_num_params(n, L, b, r);
    for (int64_t p = 0; p < 2 * P; ++p) reg += packed[p] * packed[p];
    return 0.5 * fit + 0.5 * lambda * reg;
}

/* --------------------------------------------------------------- helpers */

/* Stable grouping of entries by an integer key in [0, K): counting sort.
 * order[start[k] .. start[k+1]) lists the entries with key k in input order. */
static void group_by_key(const int64_t* key, int64_t N, int64_t K,
                         int64_t* order, int64_t* start)
{
    for (int64_t k = 0; k <= K; ++k) start[k] = 0;
    for (int64_t e = 0; e < N; ++e) start[key[e] + 1] += 1;
    for (int64_t k = 0; k < K; ++k) start[k + 1] += start[k];
    int64_t* fill = (int64_t*)malloc((size_t)(K + 1) * sizeof(int64_t));
    memcpy(fill, start, (size_t)(K + 1) * sizeof(int64_t));
    for (int64_t e = 0; e < N; ++e) order[fill[key[e]]++] = e;
    free(fill);
}

/* Solve K s = y for a Hermitian positive definite d x d matrix K (only its
 * lower triangle is read) by the Cholesky factorization K = L L^H, then
 * L z = y, L^H s = z.  K is overwritten by L.  Returns 1 if a pivot is
 * <= piv_tol (the system is then left unsolved), else 0. */
static int chol_solve(cplx* K, const cplx* y, cplx* s, int d, double piv_tol)
{
    for (int c = 0; c < d; ++c) {
        double diag = creal(K[c * d + c]);
        for (int q = 0; q < c; ++q) diag -= creal(K[c * d + q] * conj(K[c * d + q]));
        if (!(diag > piv_tol)) return 1;
        double lcc = sqrt(diag);
        K[c * d + c] = lcc;
        for (int row = c + 1; row < d; ++row) {
            cplx acc = K[row * d + c];
            for (int q = 0; q < c; ++q) acc -= K[row * d + q] * conj(K[c * d + q]);
            K[row * d + c] = acc / lcc;
        }
    }
    cplx z[BFO_MAX_R * BFO_MAX_R];
    for (int row = 0; row < d; ++row) {
        cplx acc = y[row];
        for (int q = 0; q < row; ++q) acc -= K[row * d + q] * z[q];
        z[row] = acc / creal(K[row * d + row]);
    }
    for (int row = d - 1; row >= 0; --row) {
        cplx acc = z[row];
        for (int q = row + 1; q < d; ++q) acc -= conj(K[q * d + row]) * s[q];
        s[row] = acc / creal(K[row * d + row]);
    }
    return 0;
}

/* One regularized least-squares block update (one fiber of S^1 / S^{L+2} or
 * one slice of a middle factor): given the design vectors a_e (length d) and
 * values t_e of the entries in the block, form
 *   K = sum_e conj(a_e) a_e^T + lambda I,   y = sum_e conj(a_e) t_e
 * (Alg. 1, normal-equation lines, complex form) and overwrite `target` with
 * K^{-1} y.  Returns 1 (target untouched) if K is numerically singular. */
static int block_solve(const cplx* A, const cplx* tv, int64_t cnt, int d,
                       double lambda, double ridge_rel, cplx* target)
{
    cplx* K = (cplx*)calloc((size_t)d * d, sizeof(cplx));
    cplx y[BFO_MAX_R * BFO_MAX_R], s[BFO_MAX_R * BFO_MAX_R];
    for (int p = 0; p < d; ++p) y[p] = 0;
    for (int64_t e = 0; e < cnt; ++e) {
        const cplx* a = A + e * d;
        for (int p = 0; p < d; ++p) {
            cplx ca = conj(a[p]);
            y[p] += ca * tv[e];
            for (int q = 0; q <= p; ++q) K[p * d + q] += ca * a[q];
        }
    }
    /* ridge floor (the precision form's reading of the regularization):
     * lambda is raised to ridge_rel * trace(Gram) / d when that is larger;
     * ridge_rel = 0 leaves lambda as it is */
    double gram_trace = 0.0;
    for (int p = 0; p < d; ++p) gram_trace += creal(K[p * d + p]);
    if (ridge_rel > 0.0 && ridge_rel * gram_trace / d > lambda) lambda = ridge_rel * gram_trace / d;
    double trace = 0.0;
    for (int p = 0; p < d; ++p) {
        K[p * d + p] += lambda;
        trace += creal(K[p * d + p]);
    }
    double piv_tol = lambda > 0.0 ? 0.0 : 1e-14 * trace;
    int bad = chol_solve(K, y, s, d, piv_tol);
    if (!bad)
        for (int p = 0; p < d; ++p) target[p] = s[p];
    free(K);
    return bad;
}

/* Solve every block of one factor level: for key k the entries
 * order[start[k] .. start[k+1]) (stable) form the block.  Outer levels
 * (level 0: S^1 rows, level L+1: S^{L+2} columns) use the design vector
 * env_a[e] (length r); middle levels use a_e = env_a[e] (x) env_b[e]
 * (a[p r + q] = h_p w_q, length r^2).  Block k's solution overwrites
 * target + k * d.  Blocks are independent (each has its own buffers and its
 * sums in entry order), so they may run on several threads.  Returns the
 * number of singular blocks. */
static int64_t solve_blocks(const bfo_factors* F, int level, const int64_t* order, const int64_t* start,
                            int64_t K, const cplx* env_a, const cplx* env_b, const cplx* tv_all,
                            double lambda, double ridge_rel, cplx* target)
{
    const int r = F->r;
    const int mid = level >= 1 && level <= F->L;
    const int d = mid ? r * r : r;
    int64_t maxcnt = 0;
    for (int64_t k = 0; k < K; ++k)
        if (start[k + 1] - start[k] > maxcnt) maxcnt = start[k + 1] - start[k];
    int64_t singular = 0;
#pragma omp parallel num_threads(g_threads) reduction(+ : singular)
    {
        cplx* A = (cplx*)malloc((size_t)(maxcnt > 0 ? maxcnt : 1) * d * sizeof(cplx));
        cplx* tv = (cplx*)malloc((size_t)(maxcnt > 0 ? maxcnt : 1) * sizeof(cplx));
#pragma omp for schedule(dynamic, 64)
        for (int64_t k = 0; k < K; ++k) {
            int64_t cnt = start[k + 1] - start[k];
            for (int64_t q = 0; q < cnt; ++q) {
                int64_t e = order[start[k] + q];
                if (mid) {
                    const cplx* he = env_a + e * r;
                    const cplx* we = env_b + e * r;
                    for (int p = 0; p < r; ++p)
                        for (int c = 0; c < r; ++c) A[q * d + p * r + c] = he[p] * we[c];
                } else {
                    memcpy(A + q * d, env_a + e * r, (size_t)r * sizeof(cplx));
                }
                tv[q] = tv_all[e];
            }
            singular += block_solve(A, tv, cnt, d, lambda, ridge_rel, target + k * d);
        }
        free(A);
        free(tv);
    }
    return singular;
}

/* ------------------------------------------------------------- ALS sweep */

typedef struct {
    double train_rel_err;
    double objective;
    int64_t singular;
} bfo_stats;

/* One ALS sweep (Alg. 1), in place on `packed`.
 *
 * 1. Right environments from the current factors, for every entry e=(i,j):
 *      w_L = zL(j,:),  w_{m-1} = Z^{m+1}(k_{m+1}) w_m   (m = L..1),
 *    so w_m = Z^{m+2} ... Z^{L+1} zL(j) and w_0 is the design vector of S^1
 *    (Alg. 1, the vector v of the S^1 branch).
 * 2. S^1: for each row i, solve with a_e = w_0(e); then h_1(e) = z1(i,:).
 * 3. For m = 1..L (factor S^{m+1}): for each slice k, a_e = h_m(e) (x) w_m(e),
 *    solve, store row-major in Z^{m+1}(k); then h_{m+1}(e) = h_m(e)^T Z^{m+1}(k)
 *    with the new slice (Alg. 1, the vectors u and v of the middle branch).
 * 4. S^{L+2}: for each column j, solve with a_e = h_{L+1}(e).
 * 5. Statistics on the training set with the new factors.
 * Returns the number of singular (skipped) systems. */
int64_t bfo_als_sweep_ridge(int64_t n, int L, int b, int r, double lambda, double ridge_rel,
                            double* packed, int64_t N, const int32_t* ii,
                            const int32_t* jj, const double* t, bfo_stats* st)
{
    bfo_factors F = view(n, L, b, r, packed);
    const int64_t S = F.S;
    int64_t singular = 0;
    const cplx* tv_all = (const cplx*)t;

    cplx* w = (cplx*)malloc((size_t)(L + 1) * N * r * sizeof(cplx));
    cplx* h = (cplx*)malloc((size_t)N * r * sizeof(cplx));
    cplx* hn = (cplx*)malloc((size_t)N * r * sizeof(cplx));
    int64_t* key = (int64_t*)malloc((size_t)N * sizeof(int64_t));
    int64_t* order = (int64_t*)malloc((size_t)N * sizeof(int64_t));
    int64_t kmax = (n > S ? n : S);
    int64_t* start = (int64_t*)malloc((size_t)(kmax + 1) * sizeof(int64_t));
    int d2 = r * r;

    /* 1. right environments w[m][e][:] */
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (int64_t e = 0; e < N; ++e) {
        cplx* wL = w + ((int64_t)L * N + e) * r;
        for (int c = 0; c < r; ++c) wL[c] = F.zL[(int64_t)jj[e] * r + c];
        for (int m = L; m >= 1; --m) {
            const cplx* Zk = slice_ptr(&F, m, bfo_slice_id(ii[e], jj[e], m, L, b));
            const cplx* wm = w + ((int64_t)m * N + e) * r;
            cplx* wp = w + ((int64_t)(m - 1) * N + e) * r;
            for (int a = 0; a < r; ++a) {
                cplx acc = 0;
                for (int c = 0; c < r; ++c) acc += Zk[a * r + c] * wm[c];
                wp[a] = acc;
            }
        }
    }

    /* 2. S^1 fibers, grouped by row i */
    for (int64_t e = 0; e < N; ++e) key[e] = ii[e];
    group_by_key(key, N, n, order, start);
    singular += solve_blocks(&F, 0, order, start, n, w, NULL, tv_all, lambda, ridge_rel, F.z1);
    for (int64_t e = 0; e < N; ++e)
        memcpy(h + e * r, F.z1 + (int64_t)ii[e] * r, (size_t)r * sizeof(cplx));

    /* 3. middle factors S^{m+1}, m = 1..L, grouped by slice id k_{m+1} */
    for (int m = 1; m <= L; ++m) {
        for (int64_t e = 0; e < N; ++e) key[e] = bfo_slice_id(ii[e], jj[e], m, L, b);
        group_by_key(key, N, S, order, start);
        singular += solve_blocks(&F, m, order, start, S, h, w + (int64_t)m * N * r, tv_all, lambda, ridge_rel,
                                 slice_ptr(&F, m, 0));
#pragma omp parallel for schedule(static) num_threads(g_threads)
        for (int64_t e = 0; e < N; ++e) {
            const cplx* Zk = slice_ptr(&F, m, key[e]);
            const cplx* he = h + e * r;
            for (int c = 0; c < r; ++c) {
                cplx acc = 0;
                for (int p = 0; p < r; ++p) acc += he[p] * Zk[p * r + c];
                hn[e * r + c] = acc;
            }
        }
        memcpy(h, hn, (size_t)N * r * sizeof(cplx));
    }

    /* 4. S^{L+2} fibers, grouped by column j, design h_{L+1} */
    for (int64_t e = 0; e < N; ++e) key[e] = jj[e];
    group_by_key(key, N, n, order, start);
    singular += solve_blocks(&F, L + 1, order, start, n, h, NULL, tv_all, lambda, ridge_rel, F.zL);

    free(w); free(h); free(hn); free(key); free(order); free(start);
    (void)d2;

    if (st) {
        st->train_rel_err = bfo_rel_err(n, L, b, r, packed, N, ii, jj, t);
        st->objective = bfo_objective(n, L, b, r, lambda, packed, N, ii, jj, t);
        st->singular = singular;
    }
    return singular;
}

/* One ALS sweep with the plain regularization lambda (Alg. 1). */
int64_t bfo_als_sweep(int64_t n, int L, int b, int r, double lambda,
                      double* packed, int64_t N, const int32_t* ii,
                      const int32_t* jj, const double* t, bfo_stats* st)
{
    return bfo_als_sweep_ridge(n, L, b, r, lambda, 0.0, packed, N, ii, jj, t, st);
}

/* -------------------------------------------------------------- gradient */

/* Gradient of f = 1/2 sum |x - t|^2 (+ lambda/2 ||S||^2 if include_reg) with
 * respect to every parameter, packed as df/dRe + i df/dIm (Eqs.
 * (grad_butterfly_1), (grad_butterfly_l), (grad_butterfly_last) with
 * z = x - t, complex reading):  G = sum_e (x_e - t_e) conj(da_e/ds) + lambda s.
 * Left environments h_m and right environments w_m come from the same
 * (unchanged) factors.  Writes the objective to *objective if non-NULL. */
void bfo_grad(int64_t n, int L, int b, int r, double lambda, int include_reg,
              const double* packed, int64_t N, const int32_t* ii,
              const int32_t* jj, const double* t, double* grad,
              double* objective)
{
    bfo_factors F = view(n, L, b, r, (double*)packed);
    bfo_factors G = view(n, L, b, r, grad);
    int64_t P = bfo_num_params(n, L, b, r);
    memset(grad, 0, (size_t)(2 * P) * sizeof(double));
    const cplx* tv = (const cplx*)t;
    cplx* w = (cplx*)malloc((size_t)(L + 1) * r * sizeof(cplx));
    cplx* hh = (cplx*)malloc((size_t)(L + 2) * r * sizeof(cplx));
    int64_t* ks = (int64_t*)malloc((size_t)(L + 1) * sizeof(int64_t));
    double fit = 0.0;
    for (int64_t e = 0; e < N; ++e) {
        int64_t i = ii[e], j = jj[e];
        for (int m = 1; m <= L; ++m) ks[m] = bfo_slice_id(i, j, m, L, b);
        /* right environments w_m, m = L..0 */
        for (int c = 0; c < r; ++c) w[(int64_t)L * r + c] = F.zL[j * r + c];
        for (int m = L; m >= 1; --m) {
            const cplx* Zk = slice_ptr(&F, m, ks[m]);
            for (int a = 0; a < r; ++a) {
                cplx acc = 0;
                for (int c = 0; c < r; ++c) acc += Zk[a * r + c] * w[(int64_t)m * r + c];
                w[(int64_t)(m - 1) * r + a] = acc;
            }
        }
        /* left environments h_m, m = 1..L+1 */
        for (int a = 0; a < r; ++a) hh[1 * r + a] = F.z1[i * r + a];
        for (int m = 1; m <= L; ++m) {
            const cplx* Zk = slice_ptr(&F, m, ks[m]);
            for (int c = 0; c < r; ++c) {
                cplx acc = 0;
                for (int a = 0; a < r; ++a) acc += hh[(int64_t)m * r + a] * Zk[a * r + c];
                hh[(int64_t)(m + 1) * r + c] = acc;
            }
        }
        cplx x = 0;
        for (int c = 0; c < r; ++c) x += hh[(int64_t)(L + 1) * r + c] * F.zL[j * r + c];
        cplx z = x - tv[e];
        fit += creal(z * conj(z));
        /* S^1 fiber i: design w_0 */
        for (int a = 0; a < r; ++a) G.z1[i * r + a] += z * conj(w[a]);
        /* middle slices: design h_m (x) w_m */
        for (int m = 1; m <= L; ++m) {
            cplx* Gk = slice_ptr(&G, m, ks[m]);
            for (int p = 0; p < r; ++p)
                for (int c = 0; c < r; ++c)
                    Gk[p * r + c] += z * conj(hh[(int64_t)m * r + p] * w[(int64_t)m * r + c]);
        }
        /* S^{L+2} fiber j: design h_{L+1} */
        for (int c = 0; c < r; ++c) G.zL[j * r + c] += z * conj(hh[(int64_t)(L + 1) * r + c]);
    }
    double reg = 0.0;
    for (int64_t p = 0; p < 2 * P; ++p) reg += packed[p] * packed[p];
    if (include_reg)
        for (int64_t p = 0; p < 2 * P; ++p) grad[p] += lambda * packed[p];
    if (objective) *objective = 0.5 * fit + (include_reg ? 0.5 * lambda * reg : 0.0);
    free(w); free(hh); free(ks);
}

/* ------------------------------------------------------------ initial guess */

/* Low-rank to butterfly by exact embedding (the reading used in place of
 * Alg. 2 when R = r): z1 <- A, every middle slice <- identity, zL <- B, so
 * the butterfly reproduces A B^T exactly.  A and B are n x R complex128 with
 * R <= r; columns R..r-1 of z1/zL are filled from `pad` (n x (r-R) each,
 * A-part first, then B-part), which the caller draws. */
void bfo_embed_lowrank(int64_t n, int L, int b, int r, int R, const double* A,
                       const double* B, const double* pad, double* packed)
{
    bfo_factors F = view(n, L, b, r, packed);
    const cplx* Ac = (const cplx*)A;
    const cplx* Bc = (const cplx*)B;
    const cplx* pc = (const cplx*)pad;
    int extra = r - R;
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < r; ++a) {
            F.z1[i * r + a] = a < R ? Ac[i * R + a] : pc[i * extra + (a - R)];
            F.zL[i * r + a] = a < R ? Bc[i * R + a] : pc[(n + i) * extra + (a - R)];
        }
    for (int m = 1; m <= L; ++m)
        for (int64_t k = 0; k < F.S; ++k) {
            cplx* Zk = slice_ptr(&F, m, k);
            for (int a = 0; a < r; ++a)
                for (int c = 0; c < r; ++c) Zk[a * r + c] = (a == c) ? 1.0 : 0.0;
        }
}

/* ---------------------------------------------------------------- matvec */

/* u = X(S) V for nvec vectors (Eq. (butterfly-mat-vec) computes the same
 * product by contractions in O(n log n)); here by its definition,
 * u_i = sum_j x_ij v_j with every x_ij from Eq. (BF_tensor_rep), O(n^2).
 * V is n x nvec row-major (V[j * nvec + q]), U likewise; complex128.
 * Rows are independent and each row sums over j in order. */
void bfo_matvec(int64_t n, int L, int b, int r, const double* packed, int nvec,
                const double* V, double* U)
{
    bfo_factors F = view(n, L, b, r, (double*)packed);
    const cplx* Vc = (const cplx*)V;
    cplx* Uc = (cplx*)U;
#pragma omp parallel for schedule(dynamic, 4) num_threads(g_threads)
    for (int64_t i = 0; i < n; ++i) {
        for (int q = 0; q < nvec; ++q) Uc[i * nvec + q] = 0;
        for (int64_t j = 0; j < n; ++j) {
            cplx x = eval_entry(&F, i, j);
            for (int q = 0; q < nvec; ++q) Uc[i * nvec + q] += x * Vc[j * nvec + q];
        }
    }
}
