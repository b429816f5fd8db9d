// Learned initializer: a small MLP that maps the parameters of a problem of
// one family (omega / (pi n), receiver offset h) to gauge-fixed butterfly
// factors, trained on completions the method itself produced.  It replaces
// the low-rank start (Sec. 4.2), which remains the fallback.
//
// Network: in -> hidden -> hidden -> out, GELU after the two hidden layers,
// linear output.  Weights are kept as FP32 masters (Adam state beside them)
// and used in BF16 by every forward and backward kernel; activations,
// accumulations and gradients are FP32.  Every weight matrix is stored
// input-major, Wt[k][n] (k < fan-in, n < fan-out), so a thread per output
// reads a coalesced row segment for each k.  Inputs are mapped to [-1, 1]
// by the training set's ranges; outputs are standardized per component
// (training mean and standard deviation) and the network predicts the
// standardized values.
//
// Kernels (all hand-written): layer forward, weight gradient, input gradient
// (a reduction over the fan-out in tiles, added atomically), bias gradient,
// GELU backward, MSE loss and its gradient, Adam.  No library GEMM.
#include <cuda_bf16.h>
#include <math.h>

#include <string>
#include <vector>

#include "bfc_internal.h"
#include "bfc_util.h"

struct bfc_mlp {
    int in = 0, hid = 0;
    int64_t out = 0;
    int64_t np = 0;                       // parameter count
    int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
    float *master = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    __nv_bfloat16* wb = nullptr;          // BF16 copy of the parameters (weights used in BF16)
    float *out_mean = nullptr, *out_std = nullptr;
    std::vector<double> in_lo, in_hi;
    int64_t step = 0;
    // workspace for batches of up to MAXB samples
    float *X = nullptr, *A1 = nullptr, *H1 = nullptr, *A2 = nullptr, *H2 = nullptr, *Y = nullptr;
    float *dY = nullptr, *dH2 = nullptr, *dH1 = nullptr, *T = nullptr;
    double* d_loss = nullptr;
    std::vector<void*> allocs;
    cudaStream_t stream = nullptr;
};

namespace {

constexpr int MAXB = 32;       // samples per batch inside the kernels
constexpr int FT = 256;        // threads per CTA of the per-output kernels

__device__ __forceinline__ float gelu(float a) { return 0.5f * a * (1.f + erff(a * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float a)
{
    // d/da [a Phi(a)] = Phi(a) + a phi(a)
    const float cdf = 0.5f * (1.f + erff(a * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * a * a);
    return cdf + a * pdf;
}

// A[b][n] = bias[n] + sum_k X[b][k] Wt[k][n]; H = GELU(A) when act (else H = A).
// One thread per output n for all B samples; X staged in shared memory.
__global__ void k_lin_fwd(const float* __restrict__ X, const __nv_bfloat16* __restrict__ Wt,
                          const float* __restrict__ bias, int B, int K, int64_t N, float* __restrict__ A,
                          float* __restrict__ H, int act)
{
    extern __shared__ float xs[];   // [B][K]
    for (int q = threadIdx.x; q < B * K; q += blockDim.x) xs[q] = X[q];
    __syncthreads();
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float acc[MAXB];
#pragma unroll
    for (int b = 0; b < MAXB; ++b) acc[b] = 0.f;
    for (int k = 0; k < K; ++k) {
        const float w = __bfloat162float(Wt[(int64_t)k * N + n]);
#pragma unroll
        for (int b = 0; b < MAXB; ++b)
            if (b < B) acc[b] = fmaf(xs[b * K + k], w, acc[b]);
    }
    const float bn = bias[n];
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        if (b < B) {
            const float a = acc[b] + bn;
            if (A) A[(int64_t)b * N + n] = a;
            H[(int64_t)b * N + n] = act ? gelu(a) : a;
        }
    }
}

// dWt[k][n] = sum_b X[b][k] dA[b][n];  db[n] = sum_b dA[b][n].
__global__ void k_lin_wgrad(const float* __restrict__ X, const float* __restrict__ dA, int B, int K, int64_t N,
                            float* __restrict__ dWt, float* __restrict__ db)
{
    extern __shared__ float xs[];   // [B][K]
    for (int q = threadIdx.x; q < B * K; q += blockDim.x) xs[q] = X[q];
    __syncthreads();
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float g[MAXB];
    float s = 0.f;
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        g[b] = b < B ? dA[(int64_t)b * N + n] : 0.f;
        s += g[b];
    }
    db[n] = s;
    for (int k = 0; k < K; ++k) {
        float acc = 0.f;
#pragma unroll
        for (int b = 0; b < MAXB; ++b)
            if (b < B) acc = fmaf(xs[b * K + k], g[b], acc);
        dWt[(int64_t)k * N + n] = acc;
    }
}

// dX[b][k] += sum_{n in this CTA's range} dA[b][n] Wt[k][n].  The CTA loops
// over its range of n in tiles of 32 staged in shared memory; thread k keeps
// the B partial sums of its column, added to dX atomically at the end.
// K <= blockDim.x.
__global__ void k_lin_xgrad(const float* __restrict__ dA, const __nv_bfloat16* __restrict__ Wt, int B, int K,
                            int64_t N, int64_t per_cta, float* __restrict__ dX)
{
    __shared__ float ds[MAXB][33];
    __shared__ float ws[256][33];
    const int64_t n0 = (int64_t)blockIdx.x * per_cta;
    const int64_t n1 = n0 + per_cta < N ? n0 + per_cta : N;
    const int k = threadIdx.x;
    float acc[MAXB];
#pragma unroll
    for (int b = 0; b < MAXB; ++b) acc[b] = 0.f;
    for (int64_t t0 = n0; t0 < n1; t0 += 32) {
        __syncthreads();
        for (int q = threadIdx.x; q < MAXB * 32; q += blockDim.x) {
            const int b = q / 32, nn = q % 32;
            ds[b][nn] = (b < B && t0 + nn < n1) ? dA[(int64_t)b * N + t0 + nn] : 0.f;
        }
        for (int q = threadIdx.x; q < K * 32; q += blockDim.x) {
            const int kk = q / 32, nn = q % 32;
            ws[kk][nn] = t0 + nn < n1 ? __bfloat162float(Wt[(int64_t)kk * N + t0 + nn]) : 0.f;
        }
        __syncthreads();
        if (k < K) {
#pragma unroll 4
            for (int nn = 0; nn < 32; ++nn) {
                const float w = ws[k][nn];
#pragma unroll
                for (int b = 0; b < MAXB; ++b) acc[b] = fmaf(ds[b][nn], w, acc[b]);
            }
        }
    }
    if (k < K)
        for (int b = 0; b < B; ++b) atomicAdd(&dX[b * K + k], acc[b]);
}

// dA = dH * GELU'(A) (elementwise, in place on dH)
__global__ void k_gelu_back(float* __restrict__ dH, const float* __restrict__ A, int64_t n)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) dH[q] *= gelu_grad(A[q]);
}

// loss = mean (Y - T)^2 over B x N; dY = 2 (Y - T) / (B N)
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, int64_t n, float scale,
                      float* __restrict__ dY, double* __restrict__ loss)
{
    __shared__ double red[FT];
    double s = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const float d = Y[q] - T[q];
        dY[q] = 2.f * d * scale;
        s += (double)d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] * (double)scale);
}

// Adam (Kingma and Ba) on the FP32 masters; the BF16 copy follows.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, __nv_bfloat16* __restrict__ wb, int64_t n, float lr,
                       float c1, float c2)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float gq = g[q];
    const float mq = 0.9f * m[q] + 0.1f * gq;
    const float vq = 0.999f * v[q] + 0.001f * gq * gq;
    m[q] = mq;
    v[q] = vq;
    const float wq = w[q] - lr * (mq * c1) / (sqrtf(vq * c2) + 1e-8f);
    w[q] = wq;
    wb[q] = __float2bfloat16_rn(wq);
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int64_t n)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) wb[q] = __float2bfloat16_rn(w[q]);
}

// y = mean + std * z (de-standardized prediction, FP64 out)
__global__ void k_destd(const float* __restrict__ z, const float* __restrict__ mean, const float* __restrict__ sd,
                        int B, int64_t N, double* __restrict__ y)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)B * N) return;
    const int64_t n = q % N;
    y[q] = (double)mean[n] + (double)sd[n] * (double)z[q];
}

inline unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

bfc_status mfail(bfc_status st, const std::string& msg) { return bfc::fail(nullptr, st, "mlp: " + msg); }

#define MCK(call)                                                                    \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) return mfail(BFC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

bfc_status malloc_dev(bfc_mlp* M, void** p, size_t bytes)
{
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        return mfail(BFC_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    M->allocs.push_back(*p);
    return BFC_OK;
}

// forward of a batch already in M->X (B <= MAXB); output (standardized) in M->Y
bfc_status forward_batch(bfc_mlp* M, int B)
{
    const float* P = M->master;
    const int in = M->in, hid = M->hid;
    k_lin_fwd<<<nb(hid, FT), FT, (size_t)B * in * 4, M->stream>>>(M->X, M->wb + M->oW1, P + M->ob1, B, in, hid,
                                                                  M->A1, M->H1, 1);
    k_lin_fwd<<<nb(hid, FT), FT, (size_t)B * hid * 4, M->stream>>>(M->H1, M->wb + M->oW2, P + M->ob2, B, hid, hid,
                                                                   M->A2, M->H2, 1);
    k_lin_fwd<<<nb(M->out, FT), FT, (size_t)B * hid * 4, M->stream>>>(M->H2, M->wb + M->oW3, P + M->ob3, B, hid,
                                                                      M->out, nullptr, M->Y, 0);
    MCK(cudaGetLastError());
    return BFC_OK;
}

// loss and full gradient of a batch (inputs in M->X, standardized targets in M->T)
bfc_status backward_batch(bfc_mlp* M, int B, double* loss)
{
    const int in = M->in, hid = M->hid;
    const int64_t out = M->out;
    float* G = M->grad;
    MCK(cudaMemsetAsync(M->d_loss, 0, sizeof(double), M->stream));
    const int64_t ny = (int64_t)B * out;
    k_mse<<<std::min<int64_t>(1216, nb(ny, FT)), FT, 0, M->stream>>>(M->Y, M->T, ny, 1.f / (float)ny, M->dY,
                                                                       M->d_loss);
    // layer 3
    k_lin_wgrad<<<nb(out, FT), FT, (size_t)B * hid * 4, M->stream>>>(M->H2, M->dY, B, hid, out, G + M->oW3,
                                                                     G + M->ob3);
    MCK(cudaMemsetAsync(M->dH2, 0, (size_t)B * hid * 4, M->stream));
    const int64_t per = 2048;
    k_lin_xgrad<<<nb(out, (int)per), 256, 0, M->stream>>>(M->dY, M->wb + M->oW3, B, hid, out, per, M->dH2);
    k_gelu_back<<<nb((int64_t)B * hid, FT), FT, 0, M->stream>>>(M->dH2, M->A2, (int64_t)B * hid);
    // layer 2
    k_lin_wgrad<<<nb(hid, FT), FT, (size_t)B * hid * 4, M->stream>>>(M->H1, M->dH2, B, hid, hid, G + M->oW2,
                                                                     G + M->ob2);
    MCK(cudaMemsetAsync(M->dH1, 0, (size_t)B * hid * 4, M->stream));
    k_lin_xgrad<<<nb(hid, (int)per), 256, 0, M->stream>>>(M->dH2, M->wb + M->oW2, B, hid, hid, per, M->dH1);
    k_gelu_back<<<nb((int64_t)B * hid, FT), FT, 0, M->stream>>>(M->dH1, M->A1, (int64_t)B * hid);
    // layer 1
    k_lin_wgrad<<<nb(hid, FT), FT, (size_t)B * in * 4, M->stream>>>(M->X, M->dH1, B, in, hid, G + M->oW1,
                                                                    G + M->ob1);
    MCK(cudaGetLastError());
    if (loss) {
        MCK(cudaMemcpyAsync(loss, M->d_loss, sizeof(double), cudaMemcpyDeviceToHost, M->stream));
        MCK(cudaStreamSynchronize(M->stream));
    }
    return BFC_OK;
}

// inputs -> [-1, 1] by the stored ranges, into M->X
bfc_status stage_inputs(bfc_mlp* M, int B, const double* x)
{
    std::vector<float> h((size_t)B * M->in);
    for (int b = 0; b < B; ++b)
        for (int q = 0; q < M->in; ++q) {
            const double lo = M->in_lo[q], hi = M->in_hi[q];
            const double s = hi > lo ? (x[(size_t)b * M->in + q] - lo) / (hi - lo) * 2.0 - 1.0 : 0.0;
            h[(size_t)b * M->in + q] = (float)s;
        }
    MCK(cudaMemcpyAsync(M->X, h.data(), h.size() * 4, cudaMemcpyHostToDevice, M->stream));
    MCK(cudaStreamSynchronize(M->stream));
    return BFC_OK;
}

}  // namespace

extern "C" {

bfc_status bfc_mlp_create(int32_t in_dim, int32_t hidden, int64_t out_dim, uint64_t seed, bfc_mlp** out)
{
    if (out) *out = nullptr;
    if (!out || in_dim < 1 || in_dim > 64 || hidden < 1 || hidden > 256 || out_dim < 1 ||
        out_dim > ((int64_t)1 << 31))
        return mfail(BFC_EINVAL, "need 1 <= in <= 64, 1 <= hidden <= 256, 1 <= out <= 2^31");
    bfc_mlp* M = new bfc_mlp();
    M->in = in_dim;
    M->hid = hidden;
    M->out = out_dim;
    M->oW1 = 0;
    M->ob1 = M->oW1 + (int64_t)in_dim * hidden;
    M->oW2 = M->ob1 + hidden;
    M->ob2 = M->oW2 + (int64_t)hidden * hidden;
    M->oW3 = M->ob2 + hidden;
    M->ob3 = M->oW3 + (int64_t)hidden * out_dim;
    M->np = M->ob3 + out_dim;
    M->in_lo.assign(in_dim, -1.0);
    M->in_hi.assign(in_dim, 1.0);
    bfc_status st = BFC_OK;
    auto A = [&](void** p, size_t bytes) {
        if (st == BFC_OK) st = malloc_dev(M, p, bytes);
    };
    const size_t np = (size_t)M->np;
    A((void**)&M->master, np * 4);
    A((void**)&M->m, np * 4);
    A((void**)&M->v, np * 4);
    A((void**)&M->grad, np * 4);
    A((void**)&M->wb, np * 2);
    A((void**)&M->out_mean, (size_t)out_dim * 4);
    A((void**)&M->out_std, (size_t)out_dim * 4);
    A((void**)&M->X, (size_t)MAXB * in_dim * 4);
    A((void**)&M->A1, (size_t)MAXB * hidden * 4);
    A((void**)&M->H1, (size_t)MAXB * hidden * 4);
    A((void**)&M->A2, (size_t)MAXB * hidden * 4);
    A((void**)&M->H2, (size_t)MAXB * hidden * 4);
    A((void**)&M->dH2, (size_t)MAXB * hidden * 4);
    A((void**)&M->dH1, (size_t)MAXB * hidden * 4);
    A((void**)&M->Y, (size_t)MAXB * out_dim * 4);
    A((void**)&M->dY, (size_t)MAXB * out_dim * 4);
    A((void**)&M->d_loss, sizeof(double));
    if (st == BFC_OK && cudaStreamCreateWithFlags(&M->stream, cudaStreamNonBlocking) != cudaSuccess)
        st = mfail(BFC_ECUDA, "stream");
    if (st != BFC_OK) {
        bfc_mlp_destroy(M);
        return st;
    }
    // He-normal weights from SplitMix64 + Box-Muller, zero biases
    std::vector<float> w(np, 0.f);
    uint64_t k = 0;
    auto next = [&](void) {
        k += 1;
        uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto normal = [&](void) {
        const double u1 = ((double)(next() >> 11) + 1.0) * (1.0 / 9007199254740992.0);
        const double u2 = (double)(next() >> 11) * (1.0 / 9007199254740992.0);
        return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    };
    auto fill = [&](int64_t off, int64_t cnt, int fan_in) {
        const double s = sqrt(2.0 / fan_in);
        for (int64_t q = 0; q < cnt; ++q) w[off + q] = (float)(s * normal());
    };
    fill(M->oW1, (int64_t)in_dim * hidden, in_dim);
    fill(M->oW2, (int64_t)hidden * hidden, hidden);
    fill(M->oW3, (int64_t)hidden * out_dim, hidden);
    cudaError_t e = cudaMemcpy(M->master, w.data(), np * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(M->m, 0, np * 4);
    if (e == cudaSuccess) e = cudaMemset(M->v, 0, np * 4);
    if (e == cudaSuccess) {
        std::vector<float> ones((size_t)out_dim, 1.f);
        e = cudaMemset(M->out_mean, 0, (size_t)out_dim * 4);
        if (e == cudaSuccess) e = cudaMemcpy(M->out_std, ones.data(), (size_t)out_dim * 4, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {
        k_to_bf16<<<nb(M->np, 256), 256, 0, M->stream>>>(M->master, M->wb, M->np);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
    }
    if (e != cudaSuccess) {
        bfc_mlp_destroy(M);
        return mfail(BFC_ECUDA, std::string("init: ") + cudaGetErrorString(e));
    }
    *out = M;
    return BFC_OK;
}

int64_t bfc_mlp_num_params(const bfc_mlp* M) { return M ? M->np : -1; }

void bfc_mlp_dims(const bfc_mlp* M, int32_t* in_dim, int32_t* hidden, int64_t* out_dim)
{
    if (in_dim) *in_dim = M ? M->in : 0;
    if (hidden) *hidden = M ? M->hid : 0;
    if (out_dim) *out_dim = M ? M->out : 0;
}

bfc_status bfc_mlp_set_params(bfc_mlp* M, const double* params)
{
    if (!M || !params) return mfail(BFC_EINVAL, "null argument");
    std::vector<float> w((size_t)M->np);
    for (int64_t q = 0; q < M->np; ++q) w[q] = (float)params[q];
    MCK(cudaMemcpyAsync(M->master, w.data(), w.size() * 4, cudaMemcpyHostToDevice, M->stream));
    k_to_bf16<<<nb(M->np, 256), 256, 0, M->stream>>>(M->master, M->wb, M->np);
    MCK(cudaGetLastError());
    MCK(cudaStreamSynchronize(M->stream));
    return BFC_OK;
}

bfc_status bfc_mlp_get_params(bfc_mlp* M, double* params)
{
    if (!M || !params) return mfail(BFC_EINVAL, "null argument");
    std::vector<float> w((size_t)M->np);
    MCK(cudaMemcpyAsync(w.data(), M->master, w.size() * 4, cudaMemcpyDeviceToHost, M->stream));
    MCK(cudaStreamSynchronize(M->stream));
    for (int64_t q = 0; q < M->np; ++q) params[q] = w[q];
    return BFC_OK;
}

bfc_status bfc_mlp_set_scaling(bfc_mlp* M, const double* in_lo, const double* in_hi, const double* out_mean,
                               const double* out_std)
{
    if (!M || !in_lo || !in_hi || !out_mean || !out_std) return mfail(BFC_EINVAL, "null argument");
    for (int q = 0; q < M->in; ++q) {
        if (!(in_hi[q] > in_lo[q])) return mfail(BFC_EINVAL, "input range must satisfy hi > lo");
        M->in_lo[q] = in_lo[q];
        M->in_hi[q] = in_hi[q];
    }
    std::vector<float> mu((size_t)M->out), sd((size_t)M->out);
    for (int64_t q = 0; q < M->out; ++q) {
        if (!(out_std[q] > 0.0) || !isfinite(out_mean[q])) return mfail(BFC_EINVAL, "output scale must be > 0");
        mu[q] = (float)out_mean[q];
        sd[q] = (float)out_std[q];
    }
    MCK(cudaMemcpyAsync(M->out_mean, mu.data(), mu.size() * 4, cudaMemcpyHostToDevice, M->stream));
    MCK(cudaMemcpyAsync(M->out_std, sd.data(), sd.size() * 4, cudaMemcpyHostToDevice, M->stream));
    MCK(cudaStreamSynchronize(M->stream));
    return BFC_OK;
}

bfc_status bfc_mlp_forward(bfc_mlp* M, int32_t count, const double* x, double* y)
{
    if (!M || count < 0 || (count > 0 && (!x || !y))) return mfail(BFC_EINVAL, "bad arguments");
    double* dy = nullptr;
    if (count > 0 && cudaMalloc((void**)&dy, (size_t)MAXB * M->out * 8) != cudaSuccess) {
        cudaGetLastError();
        return mfail(BFC_ENOMEM, "output buffer");
    }
    bfc_status st = BFC_OK;
    for (int32_t b0 = 0; b0 < count && st == BFC_OK; b0 += MAXB) {
        const int B = std::min<int32_t>(MAXB, count - b0);
        st = stage_inputs(M, B, x + (size_t)b0 * M->in);
        if (st == BFC_OK) st = forward_batch(M, B);
        if (st == BFC_OK) {
            k_destd<<<nb((int64_t)B * M->out, 256), 256, 0, M->stream>>>(M->Y, M->out_mean, M->out_std, B, M->out,
                                                                          dy);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(y + (size_t)b0 * M->out, dy, (size_t)B * M->out * 8, cudaMemcpyDeviceToHost,
                                    M->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
            if (e != cudaSuccess) st = mfail(BFC_ECUDA, std::string("forward: ") + cudaGetErrorString(e));
        }
    }
    cudaFree(dy);
    return st;
}

// standardized targets of `count` samples -> M->T (count <= MAXB)
static bfc_status stage_targets(bfc_mlp* M, int B, const float* tstd_dev_or_null, const double* y)
{
    if (tstd_dev_or_null) {
        MCK(cudaMemcpyAsync(M->T, tstd_dev_or_null, (size_t)B * M->out * 4, cudaMemcpyDeviceToDevice, M->stream));
        return BFC_OK;
    }
    std::vector<float> mu((size_t)M->out), sd((size_t)M->out);
    MCK(cudaMemcpyAsync(mu.data(), M->out_mean, mu.size() * 4, cudaMemcpyDeviceToHost, M->stream));
    MCK(cudaMemcpyAsync(sd.data(), M->out_std, sd.size() * 4, cudaMemcpyDeviceToHost, M->stream));
    MCK(cudaStreamSynchronize(M->stream));
    std::vector<float> t((size_t)B * M->out);
    for (int b = 0; b < B; ++b)
        for (int64_t q = 0; q < M->out; ++q)
            t[(size_t)b * M->out + q] = (float)((y[(size_t)b * M->out + q] - mu[q]) / sd[q]);
    MCK(cudaMemcpyAsync(M->T, t.data(), t.size() * 4, cudaMemcpyHostToDevice, M->stream));
    MCK(cudaStreamSynchronize(M->stream));
    return BFC_OK;
}

bfc_status bfc_mlp_grad(bfc_mlp* M, int32_t count, const double* x, const double* y, double* grads, double* loss)
{
    if (!M || count < 1 || count > MAXB || !x || !y) return mfail(BFC_EINVAL, "need 1 <= count <= 32 and data");
    if (!M->T && malloc_dev(M, (void**)&M->T, (size_t)MAXB * M->out * 4) != BFC_OK) return BFC_ENOMEM;
    BFC_TRY(stage_inputs(M, count, x));
    BFC_TRY(stage_targets(M, count, nullptr, y));
    BFC_TRY(forward_batch(M, count));
    BFC_TRY(backward_batch(M, count, loss));
    if (grads) {
        std::vector<float> g((size_t)M->np);
        MCK(cudaMemcpyAsync(g.data(), M->grad, g.size() * 4, cudaMemcpyDeviceToHost, M->stream));
        MCK(cudaStreamSynchronize(M->stream));
        for (int64_t q = 0; q < M->np; ++q) grads[q] = g[q];
    }
    return BFC_OK;
}

bfc_status bfc_mlp_train(bfc_mlp* M, int32_t count, const double* x, const double* y, int32_t epochs,
                         int32_t batch, double lr, uint64_t seed, double* loss_history)
{
    if (!M || count < 1 || !x || !y || epochs < 0 || batch < 1 || batch > MAXB || !(lr > 0.0))
        return mfail(BFC_EINVAL, "need count >= 1, epochs >= 0, 1 <= batch <= 32, lr > 0");
    const int64_t out = M->out;
    // input ranges and per-output mean / standard deviation of the training set
    std::vector<double> lo(M->in, 1e300), hi(M->in, -1e300);
    for (int32_t s = 0; s < count; ++s)
        for (int q = 0; q < M->in; ++q) {
            lo[q] = std::min(lo[q], x[(size_t)s * M->in + q]);
            hi[q] = std::max(hi[q], x[(size_t)s * M->in + q]);
        }
    for (int q = 0; q < M->in; ++q)
        if (!(hi[q] > lo[q])) { lo[q] -= 0.5; hi[q] += 0.5; }
    std::vector<double> mu((size_t)out, 0.0), sd((size_t)out, 0.0);
    for (int32_t s = 0; s < count; ++s)
        for (int64_t q = 0; q < out; ++q) mu[q] += y[(size_t)s * out + q];
    for (int64_t q = 0; q < out; ++q) mu[q] /= count;
    double sdm = 0.0;
    for (int32_t s = 0; s < count; ++s)
        for (int64_t q = 0; q < out; ++q) {
            const double d = y[(size_t)s * out + q] - mu[q];
            sd[q] += d * d;
        }
    for (int64_t q = 0; q < out; ++q) {
        sd[q] = sqrt(sd[q] / count);
        sdm += sd[q];
    }
    sdm /= (double)out;
    for (int64_t q = 0; q < out; ++q) sd[q] = std::max(sd[q], 1e-3 * sdm + 1e-30);
    BFC_TRY(bfc_mlp_set_scaling(M, lo.data(), hi.data(), mu.data(), sd.data()));
    // standardized targets on the device (FP32)
    float* Tall = nullptr;
    if (cudaMalloc((void**)&Tall, (size_t)count * out * 4) != cudaSuccess) {
        cudaGetLastError();
        return mfail(BFC_ENOMEM, "training targets");
    }
    bfc_status st = BFC_OK;
    {
        std::vector<float> t((size_t)out);
        for (int32_t s = 0; s < count && st == BFC_OK; ++s) {
            for (int64_t q = 0; q < out; ++q) t[q] = (float)((y[(size_t)s * out + q] - mu[q]) / sd[q]);
            if (cudaMemcpy(Tall + (size_t)s * out, t.data(), (size_t)out * 4, cudaMemcpyHostToDevice) != cudaSuccess)
                st = mfail(BFC_ECUDA, "target upload");
        }
    }
    if (st == BFC_OK && !M->T) st = malloc_dev(M, (void**)&M->T, (size_t)MAXB * out * 4);
    // normalized inputs of all samples (host)
    std::vector<double> xin((size_t)count * M->in);
    for (int32_t s = 0; s < count; ++s)
        for (int q = 0; q < M->in; ++q) xin[(size_t)s * M->in + q] = x[(size_t)s * M->in + q];
    std::vector<int32_t> order(count);
    for (int32_t s = 0; s < count; ++s) order[s] = s;
    uint64_t k = 0;
    auto next = [&](void) {
        k += 1;
        uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    std::vector<double> xb((size_t)MAXB * M->in);
    for (int32_t ep = 0; ep < epochs && st == BFC_OK; ++ep) {
        for (int32_t s = count - 1; s > 0; --s) std::swap(order[s], order[next() % (uint64_t)(s + 1)]);
        double lsum = 0.0;
        int nbat = 0;
        for (int32_t b0 = 0; b0 < count && st == BFC_OK; b0 += batch) {
            const int B = std::min<int32_t>(batch, count - b0);
            for (int b = 0; b < B; ++b)
                for (int q = 0; q < M->in; ++q) xb[(size_t)b * M->in + q] = xin[(size_t)order[b0 + b] * M->in + q];
            st = stage_inputs(M, B, xb.data());
            for (int b = 0; b < B && st == BFC_OK; ++b)
                if (cudaMemcpyAsync(M->T + (size_t)b * out, Tall + (size_t)order[b0 + b] * out, (size_t)out * 4,
                                    cudaMemcpyDeviceToDevice, M->stream) != cudaSuccess)
                    st = mfail(BFC_ECUDA, "batch targets");
            if (st == BFC_OK) st = forward_batch(M, B);
            double l = 0.0;
            if (st == BFC_OK) st = backward_batch(M, B, &l);
            if (st == BFC_OK) {
                M->step += 1;
                const double c1 = 1.0 / (1.0 - pow(0.9, (double)M->step));
                const double c2 = 1.0 / (1.0 - pow(0.999, (double)M->step));
                k_adam<<<nb(M->np, 256), 256, 0, M->stream>>>(M->master, M->m, M->v, M->grad, M->wb, M->np,
                                                              (float)lr, (float)c1, (float)c2);
                if (cudaGetLastError() != cudaSuccess) st = mfail(BFC_ECUDA, "adam");
            }
            lsum += l;
            ++nbat;
        }
        if (loss_history) loss_history[ep] = nbat ? lsum / nbat : 0.0;
    }
    if (st == BFC_OK && cudaStreamSynchronize(M->stream) != cudaSuccess) st = mfail(BFC_ECUDA, "train sync");
    cudaFree(Tall);
    return st;
}

void bfc_mlp_destroy(bfc_mlp* M)
{
    if (!M) return;
    if (M->stream) cudaStreamSynchronize(M->stream);
    for (void* p : M->allocs) cudaFree(p);
    if (M->stream) cudaStreamDestroy(M->stream);
    delete M;
}

}  // extern "C"
