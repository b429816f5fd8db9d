// Tensor-core (tcgen05, kind::tf32) per-slice normal equations of one middle
// level in the precision form: for every slice k of the level order,
//     K = sum_e conj(a_e) a_e^T (lower triangle),   y = sum_e conj(a_e) t_e,
// with a_e = h_e (x) w_e (a[p R + c] = h_p w_c), the left and right
// environments of entry e (Alg. 1, middle factors; Eq. (BF_tensor_rep)
// read as a linear function of one slice).  Same output record as the
// CUDA-core k_mid_gram: K packed lower-triangular, then y.
//
// Real form of the complex sums.  Write a = u + i v.  Then
//     Re K[p][q] = UU[p][q] + VV[p][q],   Im K[p][q] = UV[p][q] - VU[p][q],
//     Re y[p] = U.Re t + V.Im t,           Im y[p] = U.Im t - V.Re t,
// with UU = sum u u^T, UV = sum u v^T and so on.  Shared memory holds one
// row per real feature, u_q and v_q (128 rows), then Re t, Im t and zero
// rows up to 144, every entry one position of the contraction axis.  One
// MMA with A = rows 0..127 (M = 128) and B = rows 0..143 of the same tiles
// (N = 144) yields all of UU, UV, VU, VV and the four y products.  The rows
// are ordered so that u_p and v_p sit 16 TMEM lanes apart in one warp's
// quadrant (u_p at 32 (p / 16) + p % 16, v_p 16 rows later): at the fold a
// lane pairs its own columns with its partner's by one shuffle per column
// (the u lane keeps Re K, the v lane Im K).
//
// Precision: every operand is split into TF32 parts, x = hi + lo, and the
// product is taken as hi*hi + (lo*hi + hi*lo) (three MMAs), which keeps it to
// about FP32 accuracy.  The tensor core's FP32 accumulation into D
// truncates: every update loses about 2^-24 |D| towards zero, a bias that
// grows with the number of updates into one accumulator (measured on the
// diagonal of K: -1.2e-6 relative with all three products of two 32-entry
// chunks in one accumulator, enough to stall ALS near 1e-3 test error).  So
// every chunk of 64 entries gets its own hi*hi accumulator (at most 8
// updates), folded into per-thread Kahan sums, while the cross terms, 2^-11
// smaller, run over the whole slice in one accumulator.  The first chunk of
// a slice puts all three products into its hi*hi accumulator, so the
// cross-term accumulator of the previous slice can still be read while the
// next slice starts.  A chunk issues only the k-steps (8 entries each) that
// hold entries.
//
// Roles (one persistent CTA of 18 warps per SM; slices round-robin):
//   warp 17      loader: bulk copies of every chunk's h rows, w rows and t
//                values into a 4-stage input ring
//   warps 0..7   build the TF32 operand rows of chunk g from the ring in
//                operand stage g&1 and signal full[g&1]
//   warp 16      waits full[s] (and accempty / sempty when it reuses an
//                accumulator), issues the MMAs of the chunk, commits to
//                empty[s] and accfull
//   warps 8..15  (two per TMEM lane quadrant) fold the hi*hi accumulator of
//                every chunk into the Kahan sums once its MMAs are complete
//                (tcgen05.ld, the column blocks of the lower triangle only),
//                signal accempty, and at the end of a slice add its cross
//                terms, signal sempty and write the record (through a
//                shared-memory copy of the packed record, so the global
//                stores are coalesced)
// Every mbarrier wait is bounded; on expiry the kernel raises *err, after
// which all waits return at once (the work still runs to its end with the
// same control flow in every warp, results undefined), then waits (bounded)
// for its MMAs and copies, frees its TMEM and returns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bfc {

struct TcGram {
    static constexpr int CE = 64;                 // entries per chunk: two K blocks of 32 TF32
    static constexpr int ROWS = 144;              // u / v feature rows 0..127 | Re t 128 | Im t 129 | zeros
    static constexpr int KB = ROWS * 128;         // one K block: 144 rows x 128 B (SW128 atoms)
    static constexpr int STAGE = 4 * KB;          // [entry block][hi/lo] K blocks
    static constexpr int NCOL = 144;              // accumulator columns (N)
    static constexpr int NBIG = 2;                // per-chunk hi*hi accumulators at TMEM columns 0, 160
    static constexpr int ACC_STRIDE = 160;
    static constexpr int SMALL_COL = 320;         // per-slice cross-term accumulator
    static constexpr int TMEM_COLS = 512;
    static constexpr int NBUILD = 8;              // operand builder warps
    static constexpr int NFOLD = 8;               // fold warps: 2 per TMEM lane quadrant
    static constexpr int NTH = 32 * (NBUILD + NFOLD + 2);   // + the MMA warp + the input-loader warp
    static constexpr int RECB = (64 * 65 / 2 + 64) * 8;  // packed record copy (rank 8; a multiple of 16 bytes)
    static constexpr int SEGC = 1024;             // cached (start, end) of this CTA's first slices
    static constexpr int NIN = 4;
    static constexpr int NBARS = 9 + 2 * NIN;     // 9 pipeline barriers + 2 x NIN input-ring barriers
    static constexpr int TAIL = 256;              // barriers, TMEM slot, abort flag
    // input ring: the h and w rows and the t values of a chunk, copied in by
    // bulk copies from 16-byte-aligned starts (up to 15 leading bytes and a
    // rounded-up end: 32 bytes of slack per array)
    static constexpr int HB = CE * 8 * 8 + 32;    // rows of up to 8 complex64 values
    static constexpr int TB = CE * 8 + 32;
    static constexpr int INSTG = 2 * HB + TB;     // one ring stage (a multiple of 16 bytes)
    static constexpr size_t SMEM = 1024 + 2 * (size_t)STAGE + RECB + 8 * (size_t)SEGC + TAIL + (size_t)NIN * INSTG;
    static constexpr uint32_t WAIT_LIMIT = 1u << 22;
};
static_assert(TcGram::NBARS * 8 + 8 <= TcGram::TAIL, "barrier area");
static_assert(TcGram::RECB % 16 == 0 && TcGram::INSTG % 16 == 0 && TcGram::HB % 16 == 0, "16-byte layout");
static_assert(TcGram::SMALL_COL + TcGram::NCOL <= TcGram::TMEM_COLS &&
              TcGram::ACC_STRIDE * (TcGram::NBIG - 1) + TcGram::NCOL <= TcGram::SMALL_COL, "TMEM columns");

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle (8-row atoms of
// 1024 bytes, 16-byte chunks permuted by the row within the atom), 8-row
// groups 1024 bytes apart.  The address field is the low 14 bits (address
// >> 4), so adding (offset >> 4) to a descriptor moves it by `offset` bytes.
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;              // leading-dimension offset (not used with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride offset between 8-row groups
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}

// x = hi + lo with hi and lo TF32 numbers (10 explicit mantissa bits; the
// low 13 bits of the pattern are zero).  Each part is rounded to nearest
// (ties away from zero) by adding half a unit of the 13 dropped bits to
// the pattern and masking; x - hi is exact in FP32, so |x - hi - lo| <=
// 2^-23 |x|.
__device__ __forceinline__ void tc_split(float x, uint32_t& hi, uint32_t& lo)
{
    hi = (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
    const float r = x - __uint_as_float(hi);
    lo = (__float_as_uint(r) + 0x1000u) & 0xFFFFE000u;
}

// One potentially blocking test of an mbarrier phase: the thread may be
// suspended for up to 1 microsecond while the phase is incomplete, instead of
// spinning on issue slots the other warps need.
__device__ __forceinline__ bool tc_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the completion of phase `parity` of an mbarrier.  Returns
// at once when *abort is set; sets *abort and *err when the limit expires.
__device__ __forceinline__ void tc_wait(uint32_t bar, uint32_t parity, volatile int* abort,
                                        unsigned long long* err)
{
    if (*abort) return;
    for (uint32_t it = 0; it < TcGram::WAIT_LIMIT; ++it)
        if (tc_try_wait(bar, parity)) return;
    *abort = 1;
    atomicExch(err, 1ull);
}

__device__ __forceinline__ void tc_arrive(uint32_t bar)
{
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}

// Consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld8(uint32_t taddr, float* v)
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tc_ld2(uint32_t taddr, float* v)
{
    uint32_t r[2];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(taddr));
    v[0] = __uint_as_float(r[0]);
    v[1] = __uint_as_float(r[1]);
}

// Packed pairs of FP32 values (the f32x2 arithmetic of sm_100 and later):
// one instruction adds or subtracts two lanes' worth of values.
__device__ __forceinline__ uint64_t f2pack(float a, float b)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2unpack(uint64_t r, float& a, float& b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t f2add(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2sub(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

struct TcChunk {
    int k, base, s1;   // slice id, first entry of the chunk, end of the slice
    int idx;           // chunk index within the slice
    int sl;            // slice number within the CTA
    bool valid;
    __device__ __forceinline__ int cnt() const { return min(TcGram::CE, s1 - base); }
    __device__ __forceinline__ bool last() const { return base + TcGram::CE >= s1; }
};

// A chunk waiting for its fold: CTA chunk number, slice, and whether it
// ends the slice (then `multi`: the slice used the cross-term accumulator).
struct TcFold {
    int k, gc;
    bool valid, last, multi;
};

// Rank R <= 8 (D = R^2 <= 64 features).  Records of empty slices are zero.
template <int R>
__global__ void __launch_bounds__(TcGram::NTH, 1)
k_mid_gram_tc(const float2* __restrict__ H, const float2* __restrict__ Wm, const float2* __restrict__ tv,
              const int32_t* __restrict__ seg, float2* __restrict__ rec, int S, unsigned long long* err)
{
    static_assert(R >= 1 && R <= 8, "tensor-core Gram needs R*R <= 64");
    constexpr int D = R * R, NPK = D * (D + 1) / 2, CE = TcGram::CE, NBIG = TcGram::NBIG;
    constexpr int NF = 32 * TcGram::NFOLD;    // fold threads
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw_s = tc_smem_u32(smem_raw);
    unsigned char* ops = smem_raw + ((1024u - (raw_s & 1023u)) & 1023u);  // 2 operand stages
    float* recs = (float*)(ops + 2 * TcGram::STAGE);                       // packed record copy
    int2* segc = (int2*)((unsigned char*)recs + TcGram::RECB);             // slice bounds cache
    uint64_t* bars = (uint64_t*)(segc + TcGram::SEGC);
    uint64_t* full = bars;            // [2]     builders -> MMA warp (count NBUILD)
    uint64_t* empty = bars + 2;       // [2]     MMA commit -> builders (operand stage free)
    uint64_t* accfull = bars + 4;     // [NBIG]  MMA commit -> builders (chunk accumulated)
    uint64_t* accempty = bars + 6;    // [NBIG]  fold warps -> MMA warp (count NFOLD)
    uint64_t* sempty = bars + 8;      // [1]     fold warps read the cross terms -> MMA warp (count NFOLD)
    uint64_t* infull = bars + 9;      // [NIN]   bulk copies of a chunk's inputs landed (loader, tx bytes)
    uint64_t* inempty = bars + 9 + TcGram::NIN;   // [NIN] builders read the stage (count NBUILD)
    uint32_t* tmem_slot = (uint32_t*)(bars + TcGram::NBARS);
    volatile int* abort_s = (volatile int*)(tmem_slot + 1);
    unsigned char* inring = (unsigned char*)bars + TcGram::TAIL;           // [NIN][INSTG]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // zero both operand stages (rows never written stay zero) and the
    // records of this CTA's empty slices; cache the slice bounds
    for (int x = tid; x < 2 * TcGram::STAGE / 16; x += TcGram::NTH) ((uint4*)ops)[x] = make_uint4(0, 0, 0, 0);
    for (int k = blockIdx.x; k < S; k += gridDim.x)
        if (seg[k + 1] == seg[k])
            for (int x = tid; x < NPK + D; x += TcGram::NTH)
                rec[(size_t)k * (NPK + D) + x] = make_float2(0.f, 0.f);
    for (int i = tid; i < TcGram::SEGC; i += TcGram::NTH) {
        const int k = blockIdx.x + i * gridDim.x;
        if (k >= S) break;
        segc[i] = make_int2(seg[k], seg[k + 1]);
    }
    if (tid == 0) {
        for (int i = 0; i < TcGram::NBARS; ++i) {
            // full, inempty: one arrival per builder warp; accempty, sempty: one
            // per fold warp; empty, accfull (MMA commits), infull (loader): one
            const uint32_t cnt = (i < 2 || i >= 9 + TcGram::NIN) ? (uint32_t)TcGram::NBUILD
                                 : (i >= 6 && i < 9)             ? (uint32_t)TcGram::NFOLD
                                                                 : 1u;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem_u32(&bars[i])), "r"(cnt));
        }
        *abort_s = 0;
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(tc_smem_u32(tmem_slot)), "n"(TcGram::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // chunk enumeration (identical in every warp)
    auto first_of = [&](int k, int sl) {
        TcChunk c;
        c.valid = false;
        for (; k < S; k += gridDim.x) {
            const int i = (k - (int)blockIdx.x) / (int)gridDim.x;
            int s0, s1;
            if (i < TcGram::SEGC) {
                const int2 sb = segc[i];
                s0 = sb.x; s1 = sb.y;
            } else {
                s0 = seg[k]; s1 = seg[k + 1];
            }
            if (s1 > s0) {
                c.k = k; c.base = s0; c.s1 = s1; c.idx = 0; c.sl = sl; c.valid = true;
                break;
            }
        }
        return c;
    };
    auto advance = [&](const TcChunk& c) {
        if (!c.last()) {
            TcChunk n = c;
            n.base = c.base + CE;
            n.idx = c.idx + 1;
            return n;
        }
        return first_of(c.k + gridDim.x, c.sl + 1);
    };

    // one ring stage: h rows at 0, w rows at HB, t values at 2 HB; the byte
    // offsets of a chunk's first row inside each (the copies start at the
    // 16-byte boundary at or before it)
    auto in_off = [&](const void* base_ptr, int64_t first, int bytes_per) {
        return (int)(((uintptr_t)base_ptr + (uintptr_t)first * bytes_per) & 15u);
    };
    if (warp == TcGram::NBUILD + TcGram::NFOLD + 1) {
        // ------------------------------------------------------ loader warp
        // Bulk copies of every chunk's h rows, w rows and t values into the
        // input ring, NIN chunks ahead of the builders.
        if (lane == 0) {
            int g = 0;
            for (TcChunk c = first_of(blockIdx.x, 0); c.valid; c = advance(c), ++g) {
                const int st = g % TcGram::NIN;
                if (g >= TcGram::NIN)
                    tc_wait(tc_smem_u32(&inempty[st]), (uint32_t)((g / TcGram::NIN - 1) & 1), abort_s, err);
                if (*abort_s) break;
                unsigned char* dst = inring + (size_t)st * TcGram::INSTG;
                const int cnt = c.cnt();
                const void* srcs[3] = {H, Wm, tv};
                const int bper[3] = {R * 8, R * 8, 8};
                const int doff[3] = {0, TcGram::HB, 2 * TcGram::HB};
                uint32_t sz[3];
                uint32_t total = 0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const uintptr_t b0 = (uintptr_t)srcs[a] + (uintptr_t)c.base * bper[a];
                    const uintptr_t b1 = b0 + (uintptr_t)cnt * bper[a];
                    const uintptr_t a0 = b0 & ~(uintptr_t)15, a1 = (b1 + 15) & ~(uintptr_t)15;
                    sz[a] = (uint32_t)(a1 - a0);
                    total += sz[a];
                }
                asm volatile("{\n.reg .b64 stt;\nmbarrier.arrive.expect_tx.shared::cta.b64 stt, [%0], %1;\n}\n"
                             ::"r"(tc_smem_u32(&infull[st])), "r"(total) : "memory");
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const uintptr_t b0 = (uintptr_t)srcs[a] + (uintptr_t)c.base * bper[a];
                    const uintptr_t a0 = b0 & ~(uintptr_t)15;
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 ::"r"(tc_smem_u32(dst + doff[a])), "l"((const void*)a0), "r"(sz[a]),
                                   "r"(tc_smem_u32(&infull[st]))
                                 : "memory");
                }
            }
            // copies given up on after an abort may still land: wait for the
            // last phase issued on every stage (bounded) before the CTA exits
            for (int st = 0; st < TcGram::NIN && st < g; ++st) {
                const int last = st + ((g - 1 - st) / TcGram::NIN) * TcGram::NIN;
                for (uint32_t it = 0; it < TcGram::WAIT_LIMIT; ++it)
                    if (tc_try_wait(tc_smem_u32(&infull[st]), (uint32_t)((last / TcGram::NIN) & 1))) break;
            }
        }
        __syncwarp();
    } else if (warp == TcGram::NBUILD + TcGram::NFOLD) {
        // ------------------------------------------------------------ MMA warp
        // The first chunk of a slice puts all three products into its hi*hi
        // accumulator; later chunks send the cross terms to the slice's
        // cross-term accumulator (their truncation bias is 2^-11 smaller).
        if (lane == 0) {
            constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) |
                                       ((uint32_t)(TcGram::NCOL >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
            const uint64_t desc0 = tc_sdesc(tc_smem_u32(ops));
            int g = 0;
            for (TcChunk c = first_of(blockIdx.x, 0); c.valid; c = advance(c), ++g) {
                const int b = g & 1, bs = g % NBIG;
                tc_wait(tc_smem_u32(&full[b]), (uint32_t)((g >> 1) & 1), abort_s, err);
                if (g >= NBIG)
                    tc_wait(tc_smem_u32(&accempty[bs]), (uint32_t)((g / NBIG - 1) & 1), abort_s, err);
                if (c.idx == 1 && c.sl >= 1)
                    tc_wait(tc_smem_u32(&sempty[0]), (uint32_t)((c.sl - 1) & 1), abort_s, err);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (*abort_s) continue;
                const uint32_t d_big = tmem + (uint32_t)(bs * TcGram::ACC_STRIDE);
                const uint32_t d_small = tmem + (uint32_t)TcGram::SMALL_COL;
                const bool head = c.idx == 0;
                const int nks = (c.cnt() + 7) >> 3;   // k-steps of 8 entries that hold entries
                const uint64_t sd = desc0 + (uint64_t)((b * TcGram::STAGE) >> 4);
#pragma unroll
                for (int s8 = 0; s8 < 8; ++s8) {
                    if (s8 < nks) {
                        const int kb = s8 >> 2, ks = s8 & 3;
                        // A (rows 0..127) and B (rows 0..143) start at the same tile
                        const uint64_t hi = sd + (uint64_t)(((2 * kb) * TcGram::KB + ks * 32) >> 4);
                        const uint64_t lo = hi + (uint64_t)(TcGram::KB >> 4);
                        const uint64_t A[3] = {lo, hi, hi};
                        const uint64_t B[3] = {hi, lo, hi};
#pragma unroll
                        for (int t = 0; t < 3; ++t) {
                            // t = 2 is hi*hi, t = 0, 1 the cross terms
                            const bool big = head || t == 2;
                            const bool start = s8 == 0 && (big ? t == (head ? 0 : 2) : (c.idx == 1 && t == 0));
                            asm volatile(
                                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                                ::"r"(big ? d_big : d_small), "l"(A[t]), "l"(B[t]), "r"(IDESC),
                                "r"(start ? 0u : 1u));
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(tc_smem_u32(&empty[b]))
                             : "memory");
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(tc_smem_u32(&accfull[bs]))
                             : "memory");
            }
            if (*abort_s && g >= 1) {
                // let the issued MMAs drain (bounded) before the TMEM is freed
                for (uint32_t it = 0; it < TcGram::WAIT_LIMIT; ++it)
                    if (tc_try_wait(tc_smem_u32(&empty[(g - 1) & 1]), (uint32_t)(((g - 1) >> 1) & 1))) break;
            }
        }
        __syncwarp();
    } else if (warp >= TcGram::NBUILD) {
        // ---------------------------------------------------------- fold warps
        // Every chunk's hi*hi accumulator is folded as soon as its MMAs are
        // complete, while the builders fill the next operand stage.
        // Fold layout: warp w reads TMEM lanes 32 qd .. 32 qd + 31 (qd = w & 3):
        // lane l < 16 the row of u_p, lane l + 16 the row of v_p, p = 16 qd + l
        // % 16.  Column block c (columns 32 c .. 32 c + 31: u_q, then v_q, q =
        // 16 c .. 16 c + 15) is needed for c <= qd (lower triangle); warp half
        // hf = (w - NBUILD) >> 2 takes blocks hf and hf + 2, and hf = 1 also the
        // y columns 128 (Re t) and 129 (Im t).
        const int qd = warp & 3, hf = (warp - TcGram::NBUILD) >> 2;
        const bool is_u = lane < 16;
        const int p = 16 * qd + (lane & 15);
        const bool live = 16 * qd < D;   // some p of the quadrant is a feature
        const bool has0 = live && hf <= qd;
        const bool has1 = live && hf + 2 <= qd;
        const bool need_y = live && hf == 1;
        // Kahan sums: 8 packed pairs per column block, one scalar for y
        uint64_t sum2[2][8], comp2[2][8];
        float sum_y = 0.f, comp_y = 0.f;
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) { sum2[i][j] = 0ull; comp2[i][j] = 0ull; }

        // the u lane's Re K (own u column + partner's v column) or the v lane's
        // Im K (partner's v column - own u column)
        auto pair = [&](float own_u, float own_v) {
            const float other = __shfl_xor_sync(0xffffffffu, own_v, 16);
            return is_u ? own_u + other : other - own_u;
        };
        // half hh of a column block: v[0..7] the u columns of q = 16 c + 8 hh
        // .. + 7, v[8..15] their v columns
        auto kahan_half = [&](const float* v, int hh, uint64_t* s2, uint64_t* c2) {
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int j = 4 * hh + jj;
                const float a = pair(v[2 * jj], v[8 + 2 * jj]);
                const float b = pair(v[2 * jj + 1], v[8 + 2 * jj + 1]);
                const uint64_t y = f2sub(f2pack(a, b), c2[j]);
                const uint64_t t = f2add(s2[j], y);
                c2[j] = f2sub(f2sub(t, s2[j]), y);
                s2[j] = t;
            }
        };
        // record copy in shared memory: the u lanes write Re, the v lanes Im
        auto put_half = [&](int c, int hh, const uint64_t* s2, const uint64_t* c2, const float* w) {
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int j = 4 * hh + jj;
                float s0, s1, c0, c1;
                f2unpack(s2[j], s0, s1);
                f2unpack(c2[j], c0, c1);
                const float v2[2] = {(s0 - c0) + pair(w[2 * jj], w[8 + 2 * jj]),
                                     (s1 - c1) + pair(w[2 * jj + 1], w[8 + 2 * jj + 1])};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int q = 16 * c + 2 * j + h;
                    if (p < D && q <= p) recs[2 * (p * (p + 1) / 2 + q) + (is_u ? 0 : 1)] = (q == p && !is_u) ? 0.f : v2[h];
                }
            }
        };

        auto fold = [&](const TcFold& f) {
            const int bs = f.gc % NBIG;
            tc_wait(tc_smem_u32(&accfull[bs]), (uint32_t)((f.gc / NBIG) & 1), abort_s, err);
            __syncwarp();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t lane_base = tmem + ((uint32_t)(32 * qd) << 16);
            const uint32_t acc = lane_base + (uint32_t)(bs * TcGram::ACC_STRIDE);
            // half a column block at a time (registers)
            float v[16];
            auto ld_half = [&](uint32_t a, int hh) {
                tc_ld8(a + 8 * hh, v);
                tc_ld8(a + 16 + 8 * hh, v + 8);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            };
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                if (has0) {
                    ld_half(acc + 32 * hf, hh);
                    kahan_half(v, hh, sum2[0], comp2[0]);
                }
                if (has1) {
                    ld_half(acc + 32 * (hf + 2), hh);
                    kahan_half(v, hh, sum2[1], comp2[1]);
                }
            }
            if (need_y) {
                tc_ld2(acc + 128, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                const float y = pair(v[0], v[1]) - comp_y;
                const float t = sum_y + y;
                comp_y = (t - sum_y) - y;
                sum_y = t;
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) tc_arrive(tc_smem_u32(&accempty[bs]));
            if (!f.last) return;
            // end of the slice: add the cross terms (when the slice had more
            // than one chunk), write the record copy, release the accumulator
            const uint32_t sm = lane_base + (uint32_t)TcGram::SMALL_COL;
            auto cross_half = [&](uint32_t a, int hh) {
                if (f.multi) {
                    ld_half(a, hh);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = 0.f;
                }
            };
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                if (has0) {
                    cross_half(sm + 32 * hf, hh);
                    put_half(hf, hh, sum2[0], comp2[0], v);
                }
                if (has1) {
                    cross_half(sm + 32 * (hf + 2), hh);
                    put_half(hf + 2, hh, sum2[1], comp2[1], v);
                }
            }
            if (need_y) {
                v[0] = 0.f;
                v[1] = 0.f;
                if (f.multi) {
                    tc_ld2(sm + 128, v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                }
                const float yv = (sum_y - comp_y) + pair(v[0], v[1]);
                if (p < D) recs[2 * (NPK + p) + (is_u ? 0 : 1)] = yv;
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) tc_arrive(tc_smem_u32(&sempty[0]));
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) { sum2[i][j] = 0ull; comp2[i][j] = 0ull; }
            sum_y = 0.f;
            comp_y = 0.f;
            asm volatile("bar.sync 1, %0;" ::"n"(NF) : "memory");
            // the record (NPK + D complex values, an even count for D = R^2,
            // so records start on 16-byte boundaries) in 16-byte pieces
            const float4* src = (const float4*)recs;
            float4* out = (float4*)(rec + (size_t)f.k * (NPK + D));
            for (int x = tid - 32 * TcGram::NBUILD; x < (NPK + D) / 2; x += NF) out[x] = src[x];
            asm volatile("bar.sync 1, %0;" ::"n"(NF) : "memory");
        };

        int g = 0;
        for (TcChunk c = first_of(blockIdx.x, 0); c.valid; c = advance(c), ++g) {
            TcFold f;
            f.valid = true;
            f.k = c.k;
            f.gc = g;
            f.last = c.last();
            f.multi = c.idx > 0;
            fold(f);
        }
    } else {
        // ------------------------------------------------------- builder warps
        // operand rows of this thread: entries lane and 32 + lane (K blocks 0
        // and 1), features q = r8 + 8 j (j = 0..7) with r8 = w; the row of
        // u_q is 32 (q / 16) + q % 16 = 8 (4 (j / 2) + j % 2) + r8 and the row
        // of v_q 16 further, so the swizzled offset inside a row group is
        // fixed per thread.  Warps 0 and 1 also write Re t (row 128) and Im t
        // (row 129).
        const int r8 = warp;
        const uint32_t t_off = (uint32_t)(r8 * 128 + ((((lane >> 2) ^ r8)) << 4) + (lane & 3) * 4);
        const int rot = (lane >> 1) & 3;

        // the h_p, w_c (and t) this thread needs for chunk c, from the input
        // ring stage of the chunk (rank 8: p = j and c = r8, so one w and the
        // whole h); the stage is released to the loader once read
        constexpr int NW = R == 8 ? 1 : 8;
        struct Vals { float2 h[2][8], w[2][NW], t[2]; };
        auto load = [&](const TcChunk& c, int gc, Vals& vl) {
#pragma unroll
            for (int eb = 0; eb < 2; ++eb) {
#pragma unroll
                for (int j = 0; j < 8; ++j) vl.h[eb][j] = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < NW; ++j) vl.w[eb][j] = make_float2(0.f, 0.f);
                vl.t[eb] = make_float2(0.f, 0.f);
            }
            const int st = gc % TcGram::NIN;
            tc_wait(tc_smem_u32(&infull[st]), (uint32_t)((gc / TcGram::NIN) & 1), abort_s, err);
            const unsigned char* sb = inring + (size_t)st * TcGram::INSTG;
            const float2* hs = (const float2*)(sb + in_off(H, c.base, R * 8));
            const float2* ws = (const float2*)(sb + TcGram::HB + in_off(Wm, c.base, R * 8));
            const float2* ts = (const float2*)(sb + 2 * TcGram::HB + in_off(tv, c.base, 8));
            const int cnt = c.cnt();
#pragma unroll
            for (int eb = 0; eb < 2; ++eb) {
                const int e = 32 * eb + lane;
                if (e < cnt) {
                    if (R == 8) {
                        // the 16-byte pieces of a 64-byte row in the order
                        // rot, rot + 1, ... (mod 4): the 32 lanes then fall on
                        // 8 distinct bank groups (4 wavefronts per load instead
                        // of 16); slot j holds feature piece (j + rot) mod 4
                        const float4* hp = (const float4*)(hs + e * R);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float4 h2 = hp[(j + rot) & 3];
                            vl.h[eb][2 * j] = make_float2(h2.x, h2.y);
                            vl.h[eb][2 * j + 1] = make_float2(h2.z, h2.w);
                        }
                        vl.w[eb][0] = ws[e * R + r8];
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int q = r8 + 8 * j;
                            if (q < D) {
                                vl.h[eb][j] = hs[e * R + q / R];
                                vl.w[eb][j % NW] = ws[e * R + q % R];
                            }
                        }
                    }
                    if (warp < 2) vl.t[eb] = ts[e];
                }
            }
            __syncwarp();
            if (lane == 0) tc_arrive(tc_smem_u32(&inempty[st]));
        };

        TcChunk cur = first_of(blockIdx.x, 0);
        Vals vc;
        int g = 0;
        while (cur.valid) {
            const TcChunk nxt = advance(cur);
            load(cur, g, vc);
            const int b = g & 1;
            if (g >= 2) tc_wait(tc_smem_u32(&empty[b]), (uint32_t)(((g - 2) >> 1) & 1), abort_s, err);
            unsigned char* st = ops + b * TcGram::STAGE;
#pragma unroll
            for (int eb = 0; eb < 2; ++eb) {
                auto put = [&](uint32_t off, uint32_t hi, uint32_t lo) {
                    *(uint32_t*)(st + (2 * eb) * TcGram::KB + off) = hi;
                    *(uint32_t*)(st + (2 * eb + 1) * TcGram::KB + off) = lo;
                };
                if (warp < 2) {  // Re t at row 128, Im t at row 129 (row group 16, r8 = warp)
                    uint32_t th, tl;
                    tc_split(warp == 0 ? vc.t[eb].x : vc.t[eb].y, th, tl);
                    put(16 * 1024 + t_off, th, tl);
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    // feature q = r8 + 8 jf of slot j (rank 8: the rotated pieces)
                    const int jf = R == 8 ? 2 * (((j >> 1) + rot) & 3) + (j & 1) : j;
                    const int q = r8 + 8 * jf;
                    if (q < D) {
                        const float2 hv = vc.h[eb][j], wq = vc.w[eb][j % NW];
                        const float u = hv.x * wq.x - hv.y * wq.y;
                        const float v = hv.x * wq.y + hv.y * wq.x;
                        uint32_t uh, ul, vh, vl;
                        tc_split(u, uh, ul);
                        tc_split(v, vh, vl);
                        const uint32_t offu = (uint32_t)((4 * (jf >> 1) + (jf & 1)) * 1024) + t_off;
                        put(offu, uh, ul);          // u_q
                        put(offu + 2048, vh, vl);   // v_q, 16 rows further
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) tc_arrive(tc_smem_u32(&full[b]));
            cur = nxt;
            ++g;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TcGram::TMEM_COLS));
    }
}

}  // namespace bfc
