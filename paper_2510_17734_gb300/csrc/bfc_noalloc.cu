// bfc_residual_noalloc: residual sums of a butterfly on caller-provided
// device data, without any device allocation.  The per-block partial sums
// that the allocating paths keep in context scratch live here in one
// file-scope __device__ array of fixed size, shared by every call.
#include <mutex>

#include "bfc_internal.h"
#include "bfc_kernels.cuh"

namespace bfc {

constexpr int NOALLOC_THREADS = 256;
constexpr int64_t NOALLOC_MAX_BLOCKS = 16384;
constexpr int64_t NOALLOC_MAX_ENTRIES = NOALLOC_THREADS * NOALLOC_MAX_BLOCKS;  // 4,194,304

// [0, 2*NOALLOC_MAX_BLOCKS): per-block (sum |t - x|^2, sum |t|^2); the last
// slot is the bad-index flag.  256 KiB + 256 B, resident on every device
// that loads the library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX_BLOCKS + 32];

template <int R>
__global__ void __launch_bounds__(NOALLOC_THREADS)
k_residual_partials_noalloc(const int32_t* __restrict__ ii, const int32_t* __restrict__ jj, int64_t M, int64_t n,
                            const double2* __restrict__ z1, const double2* __restrict__ Z,
                            const double2* __restrict__ zL, int L, int b, int64_t S,
                            const double2* __restrict__ t, double* __restrict__ scratch)
{
    __shared__ double sn[NOALLOC_THREADS / 32], sd[NOALLOC_THREADS / 32];
    double num = 0.0, den = 0.0;
    const int64_t e = (int64_t)blockIdx.x * NOALLOC_THREADS + threadIdx.x;
    if (e < M) {
        const int i = ii[e], j = jj[e];
        if (i < 0 || i >= n || j < 0 || j >= n) {
            scratch[2 * NOALLOC_MAX_BLOCKS] = 1.0;  // flag: any writer sets the same value
        } else {
            const double2 x = eval_one<double, R>(i, j, z1, Z, zL, L, b, S);
            const double2 tv = t[e];
            const double dx = tv.x - x.x, dy = tv.y - x.y;
            num = dx * dx + dy * dy;
            den = tv.x * tv.x + tv.y * tv.y;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sn[threadIdx.x >> 5] = num;
        sd[threadIdx.x >> 5] = den;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int q = 0; q < NOALLOC_THREADS / 32; ++q) { a += sn[q]; c += sd[q]; }
        scratch[2 * blockIdx.x] = a;
        scratch[2 * blockIdx.x + 1] = c;
    }
}

// Fixed-order sum of the nblk partials into sums[0..1]; NaN when the flag is set.
__global__ void __launch_bounds__(256) k_residual_final_noalloc(const double* __restrict__ scratch, int64_t nblk,
                                                                double* __restrict__ sums)
{
    __shared__ double sa[256], sb[256];
    double a = 0.0, c = 0.0;
    for (int64_t q = threadIdx.x; q < nblk; q += 256) {
        a += scratch[2 * q];
        c += scratch[2 * q + 1];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = c;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) { sa[threadIdx.x] += sa[threadIdx.x + s]; sb[threadIdx.x] += sb[threadIdx.x + s]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const bool bad = scratch[2 * NOALLOC_MAX_BLOCKS] != 0.0;
        sums[0] = bad ? __longlong_as_double(0x7ff8000000000000ll) : sa[0];
        sums[1] = bad ? __longlong_as_double(0x7ff8000000000000ll) : sb[0];
    }
}

// Clears the bad-index flag at the start of every call.
__global__ void k_residual_clear_noalloc(double* __restrict__ scratch) { scratch[2 * NOALLOC_MAX_BLOCKS] = 0.0; }

// Device address of the scratch array, looked up once per device (with that
// device current) on the first call made there.  The cached address is that
// of the device's current context: the library must not be used across a
// cudaDeviceReset (a new primary context reloads the module elsewhere).
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[128];

static bfc_status noalloc_scratch(double** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, BFC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 128) return fail(nullptr, BFC_ECUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(nullptr, BFC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = (double*)p;
    }
    *out = g_noalloc_ptr[dev];
    return BFC_OK;
}

// EINVAL unless p is device or managed memory usable on the current device
// and `align`-byte aligned (cudaPointerGetAttributes allocates nothing).
static bfc_status check_device_ptr(const void* p, size_t align, const char* what)
{
    if ((uintptr_t)p % align != 0)
        return fail(nullptr, BFC_EINVAL, std::string(what) + " is not " + std::to_string(align) + "-byte aligned");
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, BFC_EINVAL, std::string(what) + ": not a CUDA pointer (" + cudaGetErrorString(e) + ")");
    }
    int dev = -1;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, BFC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (a.type == cudaMemoryTypeManaged) return BFC_OK;
    if (a.type != cudaMemoryTypeDevice)
        return fail(nullptr, BFC_EINVAL, std::string(what) + " is not device memory");
    if (a.device != dev)
        return fail(nullptr, BFC_EINVAL, std::string(what) + " is memory of another device");
    return BFC_OK;
}

template <int R>
static void launch_noalloc(int64_t n, int L, int b, const double2* F, int64_t m, const int32_t* i, const int32_t* j,
                           const double2* t, double* sums, double* scratch, cudaStream_t st)
{
    const int64_t S = (int64_t)1 << (L + 1);
    const double2* z1 = F;
    const double2* Z = F + n * R;
    const double2* zL = Z + (int64_t)L * S * R * R;
    const int64_t nblk = (m + NOALLOC_THREADS - 1) / NOALLOC_THREADS;
    k_residual_clear_noalloc<<<1, 1, 0, st>>>(scratch);
    k_residual_partials_noalloc<R><<<(unsigned)nblk, NOALLOC_THREADS, 0, st>>>(i, j, m, n, z1, Z, zL, L, b, S, t,
                                                                              scratch);
    k_residual_final_noalloc<<<1, 256, 0, st>>>(scratch, nblk, sums);
}

}  // namespace bfc

using namespace bfc;

extern "C" bfc_status bfc_residual_noalloc(int64_t n, int32_t L, int32_t b, int32_t r, const double* factors,
                                           int64_t m, const int32_t* i, const int32_t* j, const double* t,
                                           double* sums, void* stream)
{
    if (L < 0 || L > 24 || b < 1 || n < 1 || n != (int64_t)b << L || n > ((int64_t)1 << 30))
        return fail(nullptr, BFC_EINVAL, "invalid sizes: need n = b * 2^L, 0 <= L <= 24");
    if (r < 1 || r > 10) return fail(nullptr, BFC_EINVAL, "rank must be in [1, 10]");
    if (m < 0 || m > NOALLOC_MAX_ENTRIES)
        return fail(nullptr, BFC_EINVAL,
                    "m = " + std::to_string(m) + " is outside [0, " + std::to_string(NOALLOC_MAX_ENTRIES) +
                        "], the capacity of the fixed scratch of bfc_residual_noalloc");
    if (!sums || (m > 0 && (!factors || !i || !j || !t))) return fail(nullptr, BFC_EINVAL, "null argument");
    // every pointer must be device (or managed) memory of the current device
    // and aligned for the kernels' vector loads: complex128 values are read
    // as 16-byte double2, indices as int32, sums written as doubles
    BFC_TRY(check_device_ptr(sums, 8, "sums"));
    if (m > 0) {
        BFC_TRY(check_device_ptr(factors, 16, "factors"));
        BFC_TRY(check_device_ptr(t, 16, "t"));
        BFC_TRY(check_device_ptr(i, 4, "i"));
        BFC_TRY(check_device_ptr(j, 4, "j"));
    }
    cudaStream_t st = (cudaStream_t)stream;
    double* scratch = nullptr;
    BFC_TRY(noalloc_scratch(&scratch));
    if (m == 0) {
        cudaError_t e = cudaMemsetAsync(sums, 0, 2 * sizeof(double), st);
        if (e != cudaSuccess) return fail(nullptr, BFC_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
        return BFC_OK;
    }
    const double2* F = (const double2*)factors;
    const double2* tv = (const double2*)t;
    switch (r) {
    case 1: launch_noalloc<1>(n, L, b, F, m, i, j, tv, sums, scratch, st); break;
    case 2: launch_noalloc<2>(n, L, b, F, m, i, j, tv, sums, scratch, st); break;
    case 3: launch_noalloc<3>(n, L, b, F, m, i, j, tv, sums, scratch, st); break;
    case 4: launch_noalloc<4>(n, L, b, F, m, i, j, tv, sums, scratch, st); break;
    case 5: launch_noalloc<5>(n, L, b, F, m, i, j, tv, sums, scratch, st); break;
    case 6: launch_noalloc<6>(n, L, b, F, m, i, j, tv, sums, scratch, st); break;
    case 7: launch_noalloc<7>(n, L, b, F, m, i, j, tv, sums, scratch, st); break;
    case 8: launch_noalloc<8>(n, L, b, F, m, i, j, tv, sums, scratch, st); break;
    case 9: launch_noalloc<9>(n, L, b, F, m, i, j, tv, sums, scratch, st); break;
    default: launch_noalloc<10>(n, L, b, F, m, i, j, tv, sums, scratch, st); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, BFC_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return BFC_OK;
}
