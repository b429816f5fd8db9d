// Non-templated kernels of libbfc: the once-per-Omega preparation (a stable
// LSD radix sort of the entries by the key of each factor level, segment
// offsets and position maps -- the "transpose the sparse tensor according to
// the index being solved for" step of App. A.2), deterministic reductions,
// conversions and the low-rank embedding.
#include "bfc_util.h"

namespace bfc {

// ---------------------------------------------------------------- keys

// Level key of every entry: l = 0 row i, l = L+1 column j, otherwise the
// slice id psi^{-1}(i_0..i_{L-m}, j_0..j_{m-1}) of S^{m+1}, m = l.
// Sort key of every entry for one level: the row, the slice id of S^{level+1}
// or the column.  With loc > 0 (middle levels) the key is composite,
// slice * loc + (row or column index within the slice's block, i mod loc or
// j mod loc), so that inside a slice the entries of one row (or column) are
// contiguous.
__global__ void k_level_keys(const int32_t* __restrict__ ii, const int32_t* __restrict__ jj, int64_t N,
                             int level, int L, int b, int64_t loc, int by_col, uint32_t* __restrict__ key,
                             int32_t* __restrict__ idx)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int i = ii[e], j = jj[e];
    uint32_t k;
    if (level == 0) k = (uint32_t)i;
    else if (level == L + 1) k = (uint32_t)j;
    else {
        const int m = level, pi = i / b, pj = j / b;
        k = (uint32_t)(((pi >> (m - 1)) << m) | (pj >> (L - m)));
        if (loc > 0) k = (uint32_t)((int64_t)k * loc + (by_col ? j % loc : i % loc));
    }
    key[e] = k;
    idx[e] = (int32_t)e;
}

// All level keys of m pairs: keys[e * (L+2) + l] (the same key function the
// sort uses).
__global__ void k_all_keys(const int32_t* __restrict__ ii, const int32_t* __restrict__ jj, int64_t M, int L,
                           int b, int32_t* __restrict__ keys)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M) return;
    const int i = ii[e], j = jj[e], pi = i / b, pj = j / b;
    int32_t* out = keys + e * (L + 2);
    out[0] = i;
    for (int m = 1; m <= L; ++m) out[m] = ((pi >> (m - 1)) << m) | (pj >> (L - m));
    out[L + 1] = j;
}

// ---------------------------------------------------------- radix sort
// One 8-bit digit per pass, tiles of RS_TILE consecutive elements.  A pass
// counts digits per tile (digit-major table), scans the table, and scatters
// each tile in order: the rank of an element among equal digits of its tile
// is (count in earlier warps) + (earlier lanes of its warp), so every pass is
// stable and the whole sort is deterministic.

__global__ void __launch_bounds__(RS_TILE) k_rs_count(const uint32_t* __restrict__ keys, int64_t N, int shift,
                                                      int64_t T, int32_t* __restrict__ counts)
{
    __shared__ int32_t h[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0;
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * RS_TILE + threadIdx.x;
    if (e < N) atomicAdd(&h[(keys[e] >> shift) & 255u], 1);
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += blockDim.x) counts[(int64_t)t * T + blockIdx.x] = h[t];
}

// Exclusive scan of M int32 values in place, one block of 1024 threads:
// each thread owns a contiguous chunk.
__global__ void __launch_bounds__(1024) k_scan_excl(int32_t* __restrict__ data, int64_t M)
{
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int64_t per = (M + 1023) / 1024;
    const int64_t lo = (int64_t)t * per, hi = min(M, lo + per);
    int64_t s = 0;
    for (int64_t q = lo; q < hi; ++q) s += data[q];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        int64_t run = 0;
        for (int q = 0; q < 1024; ++q) { int64_t v = part[q]; part[q] = run; run += v; }
    }
    __syncthreads();
    int64_t run = part[t];
    for (int64_t q = lo; q < hi; ++q) { int32_t v = data[q]; data[q] = (int32_t)run; run += v; }
}

__global__ void __launch_bounds__(RS_TILE) k_rs_scatter(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin,
                                                        uint32_t* __restrict__ kout, int32_t* __restrict__ vout,
                                                        int64_t N, int shift, int64_t T,
                                                        const int32_t* __restrict__ offs)
{
    __shared__ int32_t cnt[RS_TILE / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int q = tid; q < (RS_TILE / 32) * 256; q += blockDim.x) (&cnt[0][0])[q] = 0;
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * RS_TILE + tid;
    const bool valid = e < N;
    const uint32_t key = valid ? kin[e] : 0u;
    const int32_t val = valid ? vin[e] : 0;
    const int digit = valid ? (int)((key >> shift) & 255u) : 256 + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const int leader = __ffs(peers) - 1;
    if (valid && lane == leader) cnt[warp][digit] = __popc(peers);
    __syncthreads();
    if (tid < 256) {
        int32_t run = 0;
        for (int w = 0; w < RS_TILE / 32; ++w) { int32_t c = cnt[w][tid]; cnt[w][tid] = run; run += c; }
    }
    __syncthreads();
    if (valid) {
        const int rank = cnt[warp][digit] + __popc(peers & ((1u << lane) - 1u));
        const int64_t pos = (int64_t)offs[(int64_t)digit * T + blockIdx.x] + rank;
        kout[pos] = key;
        vout[pos] = val;
    }
}

// seg[k] = first position whose sorted key is >= k, seg[K] = N.
// Segment offsets of the sorted keys (key / div is the segment id, K segments).
__global__ void k_segments(const uint32_t* __restrict__ skeys, int64_t N, int64_t K, int64_t div,
                           int32_t* __restrict__ seg)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int64_t kp = (int64_t)skeys[p] / div;
    const int64_t kprev = p ? (int64_t)skeys[p - 1] / div : -1;
    for (int64_t k = kprev + 1; k <= kp; ++k) seg[k] = (int32_t)p;
    if (p == N - 1)
        for (int64_t k = kp + 1; k <= K; ++k) seg[k] = (int32_t)N;
}

__global__ void k_invert(const int32_t* __restrict__ perm, int64_t N, int32_t* __restrict__ pos)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) pos[perm[p]] = (int32_t)p;
}

// out[p] = pos_other[perm[p]]
__global__ void k_compose(const int32_t* __restrict__ perm, const int32_t* __restrict__ pos_other, int64_t N,
                          int32_t* __restrict__ out)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) out[p] = pos_other[perm[p]];
}

__global__ void k_gather_i32(const int32_t* __restrict__ src, const int32_t* __restrict__ perm, int64_t N,
                             int32_t* __restrict__ out)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) out[p] = src[perm[p]];
}

__global__ void k_gather_c_f(const double2* __restrict__ src, const int32_t* __restrict__ perm, int64_t N,
                             float2* __restrict__ out)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) {
        const double2 v = src[perm[p]];
        out[p] = make_float2((float)v.x, (float)v.y);
    }
}

__global__ void k_gather_c_d(const double2* __restrict__ src, const int32_t* __restrict__ perm, int64_t N,
                             double2* __restrict__ out)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) out[p] = src[perm[p]];
}

// ---------------------------------------------------------- utilities

__global__ void k_d2f(const double2* __restrict__ src, float2* __restrict__ dst, int64_t n)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) dst[p] = make_float2((float)src[p].x, (float)src[p].y);
}

// Index range and duplicate-free check helpers: flag[0] |= 1 on an index
// outside [0, n), flag[0] |= 2 on a NaN/Inf value.
__global__ void k_check_entries(const int32_t* __restrict__ ii, const int32_t* __restrict__ jj,
                                const double2* __restrict__ t, int64_t M, int64_t n, int* __restrict__ flag)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M) return;
    const int i = ii[e], j = jj[e];
    if (i < 0 || i >= n || j < 0 || j >= n) atomicOr(flag, 1);
    if (t) {
        const double2 v = t[e];
        if (!isfinite(v.x) || !isfinite(v.y)) atomicOr(flag, 2);
    }
}

// Duplicate (i, j) pairs: in row order every row segment must hold distinct
// columns.  One warp per row compares each entry with the later ones of its
// row; flag[0] |= 4 on a duplicate.
__global__ void k_row_dups(const int32_t* __restrict__ seg, const int32_t* __restrict__ jrow, int64_t nrows,
                           int* __restrict__ flag)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= nrows) return;
    const int s0 = seg[row], s1 = seg[row + 1];
    bool dup = false;
    for (int p = s0 + lane; p < s1 && !dup; p += 32) {
        const int jp = jrow[p];
        for (int q = p + 1; q < s1; ++q)
            if (jrow[q] == jp) { dup = true; break; }
    }
    if (__any_sync(0xffffffffu, dup) && lane == 0) atomicOr(flag, 4);
}

// Deterministic reductions: one block, fixed assignment and order.
__global__ void __launch_bounds__(1024) k_reduce_pairs(const double* __restrict__ part, int64_t count,
                                                       double* __restrict__ out)
{
    __shared__ double sa[1024], sb[1024];
    double a = 0.0, b = 0.0;
    for (int64_t q = threadIdx.x; q < count; q += blockDim.x) {
        a += part[2 * q];
        b += part[2 * q + 1];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) { sa[threadIdx.x] += sa[threadIdx.x + s]; sb[threadIdx.x] += sb[threadIdx.x + s]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = sa[0]; out[1] = sb[0]; }
}

__global__ void __launch_bounds__(1024) k_reduce_single(const double* __restrict__ part, int64_t count,
                                                        double* __restrict__ out)
{
    __shared__ double sa[1024];
    double a = 0.0;
    for (int64_t q = threadIdx.x; q < count; q += blockDim.x) a += part[q];
    sa[threadIdx.x] = a;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sa[threadIdx.x] += sa[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sa[0];
}

// Per-block sum of squares of a complex128 vector (block partials in part).
__global__ void __launch_bounds__(256) k_sumsq(const double2* __restrict__ x, int64_t n, double* __restrict__ part)
{
    __shared__ double sw[8];
    double a = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = x[q];
        a += v.x * v.x + v.y * v.y;
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += sw[q];
        part[blockIdx.x] = s;
    }
}

// y += alpha * x (complex128 vectors viewed as doubles)
__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, double alpha, int64_t n)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) y[q] += alpha * x[q];
}

// Exact embedding of a rank-R low-rank pair (A, B: n x R) into butterfly
// factors of rank r >= R: z1 = [A 0], every middle slice = I_r, zL = [B 0].
__global__ void k_embed(const double2* __restrict__ A, const double2* __restrict__ B, int64_t n, int R, int r,
                        int64_t nslices, double2* __restrict__ z1, double2* __restrict__ Z, double2* __restrict__ zL)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nr = n * r;
    if (q < nr) {
        const int64_t i = q / r;
        const int a = (int)(q - i * r);
        z1[q] = a < R ? A[i * R + a] : make_double2(0.0, 0.0);
        zL[q] = a < R ? B[i * R + a] : make_double2(0.0, 0.0);
    }
    const int64_t nz = nslices * r * r;
    if (q < nz) {
        const int64_t w = q % ((int64_t)r * r);
        const int a = (int)(w / r), c = (int)(w % r);
        Z[q] = make_double2(a == c ? 1.0 : 0.0, 0.0);
    }
}

// Per-block partial dot products of two double vectors (deterministic order).
__global__ void __launch_bounds__(256) k_dot(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                                             double* __restrict__ part)
{
    __shared__ double sw[8];
    double s = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        s += a[q] * b[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sw[q];
        part[blockIdx.x] = t;
    }
}

// y = a x + b z
__global__ void k_axpby(double* __restrict__ y, double a, const double* __restrict__ x, double b,
                        const double* __restrict__ z, int64_t n)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) y[q] = a * x[q] + b * z[q];
}

// ------------------------------------------------------------ launchers

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t sort_level(const int32_t* d_i, const int32_t* d_j, int64_t N, int level, int L, int b,
                       int64_t K, int64_t loc, int by_col, cudaStream_t st, SortScratch& s, int32_t* perm_out,
                       int32_t* seg_out, uint32_t** sorted_keys)
{
    k_level_keys<<<nblk(N, 256), 256, 0, st>>>(d_i, d_j, N, level, L, b, loc, by_col, s.k0, s.v0);
    const int64_t KK = loc > 0 ? K * loc : K;
    int bits = 0;
    while (((int64_t)1 << bits) < KK) ++bits;
    const int passes = (bits + 7) / 8;
    const int64_t T = (N + RS_TILE - 1) / RS_TILE;
    uint32_t *ka = s.k0, *kb = s.k1;
    int32_t *va = s.v0, *vb = s.v1;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        k_rs_count<<<(unsigned)T, RS_TILE, 0, st>>>(ka, N, shift, T, s.counts);
        k_scan_excl<<<1, 1024, 0, st>>>(s.counts, 256 * T);
        k_rs_scatter<<<(unsigned)T, RS_TILE, 0, st>>>(ka, va, kb, vb, N, shift, T, s.counts);
        uint32_t* tk = ka; ka = kb; kb = tk;
        int32_t* tv = va; va = vb; vb = tv;
    }
    k_segments<<<nblk(N, 256), 256, 0, st>>>(ka, N, K, loc > 0 ? loc : 1, seg_out);
    cudaMemcpyAsync(perm_out, va, (size_t)N * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (sorted_keys) *sorted_keys = ka;
    return cudaGetLastError();
}

void launch_all_keys(const int32_t* ii, const int32_t* jj, int64_t M, int L, int b, int32_t* keys,
                     cudaStream_t st)
{
    k_all_keys<<<nblk(M, 256), 256, 0, st>>>(ii, jj, M, L, b, keys);
}
void launch_dot(const double* a, const double* b, int64_t n, double* part, int nblocks, double* out,
                cudaStream_t st)
{
    k_dot<<<nblocks, 256, 0, st>>>(a, b, n, part);
    k_reduce_single<<<1, 1024, 0, st>>>(part, nblocks, out);
}
void launch_axpby(double* y, double a, const double* x, double b, const double* z, int64_t n, cudaStream_t st)
{
    if (n > 0) k_axpby<<<nblk(n, 256), 256, 0, st>>>(y, a, x, b, z, n);
}
void launch_invert(const int32_t* perm, int64_t N, int32_t* pos, cudaStream_t st)
{
    k_invert<<<nblk(N, 256), 256, 0, st>>>(perm, N, pos);
}
void launch_compose(const int32_t* perm, const int32_t* pos_other, int64_t N, int32_t* out, cudaStream_t st)
{
    k_compose<<<nblk(N, 256), 256, 0, st>>>(perm, pos_other, N, out);
}
void launch_gather_i32(const int32_t* src, const int32_t* perm, int64_t N, int32_t* out, cudaStream_t st)
{
    k_gather_i32<<<nblk(N, 256), 256, 0, st>>>(src, perm, N, out);
}
void launch_gather_values(const double2* src, const int32_t* perm, int64_t N, void* out, bool fp32,
                          cudaStream_t st)
{
    if (fp32) k_gather_c_f<<<nblk(N, 256), 256, 0, st>>>(src, perm, N, (float2*)out);
    else k_gather_c_d<<<nblk(N, 256), 256, 0, st>>>(src, perm, N, (double2*)out);
}
void launch_d2f(const double2* src, float2* dst, int64_t n, cudaStream_t st)
{
    if (n > 0) k_d2f<<<nblk(n, 256), 256, 0, st>>>(src, dst, n);
}
void launch_check_entries(const int32_t* ii, const int32_t* jj, const double2* t, int64_t M, int64_t n,
                          int* flag, cudaStream_t st)
{
    if (M > 0) k_check_entries<<<nblk(M, 256), 256, 0, st>>>(ii, jj, t, M, n, flag);
}
void launch_row_dups(const int32_t* seg, const int32_t* jrow, int64_t nrows, int* flag, cudaStream_t st)
{
    k_row_dups<<<nblk(nrows, 8), 256, 0, st>>>(seg, jrow, nrows, flag);
}
void launch_reduce_pairs(const double* part, int64_t count, double* out, cudaStream_t st)
{
    k_reduce_pairs<<<1, 1024, 0, st>>>(part, count, out);
}
void launch_reduce_single(const double* part, int64_t count, double* out, cudaStream_t st)
{
    k_reduce_single<<<1, 1024, 0, st>>>(part, count, out);
}
void launch_sumsq(const double2* x, int64_t n, double* part, int nblocks, cudaStream_t st)
{
    k_sumsq<<<nblocks, 256, 0, st>>>(x, n, part);
}
void launch_axpy(double* y, const double* x, double alpha, int64_t n, cudaStream_t st)
{
    if (n > 0) k_axpy<<<nblk(n, 256), 256, 0, st>>>(y, x, alpha, n);
}
void launch_embed(const double2* A, const double2* B, int64_t n, int R, int r, int64_t nslices, double2* z1,
                  double2* Z, double2* zL, cudaStream_t st)
{
    const int64_t m = n * r > nslices * r * r ? n * r : nslices * r * r;
    k_embed<<<nblk(m, 256), 256, 0, st>>>(A, B, n, R, r, nslices, z1, Z, zL);
}

}  // namespace bfc
