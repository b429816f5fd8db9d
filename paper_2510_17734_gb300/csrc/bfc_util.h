// Launchers of the non-templated kernels (bfc_util.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bfc {

constexpr int RS_TILE = 1024;

// Scratch of the level sorts: keys / values ping-pong and the digit table.
struct SortScratch {
    uint32_t *k0 = nullptr, *k1 = nullptr;
    int32_t *v0 = nullptr, *v1 = nullptr;
    int32_t* counts = nullptr;   // 256 * ceil(N / RS_TILE)
};

// Stable sort of the entries by the key of `level` (K distinct key values):
// perm_out[p] = entry at position p, seg_out[k] = first position of key k
// (K + 1 values).
// loc > 0 (middle levels): inside a slice, the entries are ordered by their
// row (by_col = 0: i mod loc) or column (j mod loc) within the slice's block;
// *sorted_keys (may be NULL) receives the device array of sorted keys (in s).
cudaError_t sort_level(const int32_t* d_i, const int32_t* d_j, int64_t N, int level, int L, int b,
                       int64_t K, int64_t loc, int by_col, cudaStream_t st, SortScratch& s, int32_t* perm_out,
                       int32_t* seg_out, uint32_t** sorted_keys);

void launch_all_keys(const int32_t* ii, const int32_t* jj, int64_t M, int L, int b, int32_t* keys,
                     cudaStream_t st);
void launch_dot(const double* a, const double* b, int64_t n, double* part, int nblocks, double* out,
                cudaStream_t st);
void launch_axpby(double* y, double a, const double* x, double b, const double* z, int64_t n, cudaStream_t st);
void launch_invert(const int32_t* perm, int64_t N, int32_t* pos, cudaStream_t st);
void launch_compose(const int32_t* perm, const int32_t* pos_other, int64_t N, int32_t* out, cudaStream_t st);
void launch_gather_i32(const int32_t* src, const int32_t* perm, int64_t N, int32_t* out, cudaStream_t st);
void launch_gather_values(const double2* src, const int32_t* perm, int64_t N, void* out, bool fp32,
                          cudaStream_t st);
void launch_d2f(const double2* src, float2* dst, int64_t n, cudaStream_t st);
void launch_check_entries(const int32_t* ii, const int32_t* jj, const double2* t, int64_t M, int64_t n,
                          int* flag, cudaStream_t st);
void launch_row_dups(const int32_t* seg, const int32_t* jrow, int64_t nrows, int* flag, cudaStream_t st);
void launch_reduce_pairs(const double* part, int64_t count, double* out, cudaStream_t st);
void launch_reduce_single(const double* part, int64_t count, double* out, cudaStream_t st);
void launch_sumsq(const double2* x, int64_t n, double* part, int nblocks, cudaStream_t st);
void launch_axpy(double* y, const double* x, double alpha, int64_t n, cudaStream_t st);
void launch_embed(const double2* A, const double2* B, int64_t n, int R, int r, int64_t nslices, double2* z1,
                  double2* Z, double2* zL, cudaStream_t st);

// Left-orthogonal gauge of the FP64 factors (bfc_gauge.cu).
// Randomized low-rank to butterfly conversion (Alg. 2, bfc_lr2bf.cu): the
// Gaussian count it reads (O_0, then the left and right levels), its scratch
// size and the launch sequence into the FP64 factors.
inline int64_t lr2bf_gaussian_count(int64_t n, int L, int b, int r, int p)
{
    const int H = L / 2;
    int64_t rows = n;
    for (int l = 1; l <= H; ++l) rows += (int64_t)b << (L - l);
    for (int l = 1; l <= L - H; ++l) rows += (int64_t)b << (L - l);
    return rows * (r + p);
}
size_t lr2bf_scratch_bytes(int64_t n, int L, int b, int R, int r, int p);
cudaError_t lr2bf_run(const double2* A, const double2* B, const double2* Gs, int64_t n, int L, int b, int R, int r,
                      int p, double2* z1, double2* Z, double2* zL, void* scratch, cudaStream_t st);

// One level of it (0 = the leaf blocks of z1, m = 1..L = the slice pairs of
// S^{m+1}); ADF (Alg. 5) moves the orthogonality centre with it.
cudaError_t launch_canon_level(double2* z1, double2* Z, double2* zL, int64_t n, int L, int b, int r, int level,
                               cudaStream_t st);
// Right-to-left orthogonalization (App. A.3, mirrored): every factor but z1
// right-orthonormal, entries unchanged.
cudaError_t launch_rl_orthogonalize(double2* z1, double2* Z, double2* zL, int64_t n, int L, int b, int r,
                                    cudaStream_t st);
cudaError_t launch_canonicalize(double2* z1, double2* Z, double2* zL, int64_t n, int L, int b, int r,
                                cudaStream_t st);

}  // namespace bfc
