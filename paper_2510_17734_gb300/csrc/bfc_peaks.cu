// Measured arithmetic peaks of the current device: dependent-FMA chains (eight
// independent chains per thread, 256 threads per CTA, eight CTAs per SM) in
// FP32 and in FP64, best of five timed launches.  They are the denominators
// of the ALU rooflines of the CUDA-core kernels (the Gram on CUDA cores is
// FP32-bound, the FP64 solves FP64-bound).
#include "bfc_internal.h"

namespace {

template <typename T>
__global__ void k_fma_chain(T* out, int iters, T a, T b)
{
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x * 1e-3) + (T)k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
        }
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
cudaError_t time_chain(int blocks, int iters, T* out, double* tflops)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0);
        k_fma_chain<T><<<blocks, 256>>>(out, iters, (T)0.9999, (T)1e-5);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && e == cudaSuccess && ms < best) best = ms;   // first launch is a warm-up
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e == cudaSuccess) *tflops = 2.0 * 8 * 16 * (double)iters * blocks * 256 / (best * 1e-3) / 1e12;
    return e;
}

}  // namespace

extern "C" bfc_status bfc_measure_alu_peaks(double* fp32_tflops, double* fp64_tflops)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void* buf = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&buf, (size_t)sms * 8 * 256 * sizeof(double));
    double f32 = 0.0, f64 = 0.0;
    if (e == cudaSuccess) e = time_chain<float>(sms * 8, 4000, (float*)buf, &f32);
    if (e == cudaSuccess) e = time_chain<double>(sms * 8, 200, (double*)buf, &f64);
    if (buf) cudaFree(buf);
    if (e != cudaSuccess) return bfc::fail(nullptr, BFC_ECUDA, std::string("peaks: ") + cudaGetErrorString(e));
    if (fp32_tflops) *fp32_tflops = f32;
    if (fp64_tflops) *fp64_tflops = f64;
    return BFC_OK;
}
