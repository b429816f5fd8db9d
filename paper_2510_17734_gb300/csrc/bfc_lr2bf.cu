// Randomized low-rank to butterfly conversion (Alg. 2, Sec. 4.2), FP64 on the
// master factors.  Input X = A B^T (A, B: n x R), the Gaussian sketch
// matrices (caller-drawn), oversampling p; C = r + p sketch columns.
//
// 1. Outer sketches M = A (B^T O_0), N = B (A^T O_0).  For every leaf block,
//    QR with column pivoting of its b rows of M (of N): the first r columns of
//    Q are the rows z1[i] (zL[j]) of the block, V = Q^H A(block) (W =
//    Q^H B(block)) its r x R coefficients.
// 2. Left levels l = 1 .. H (H = floor(L / 2)): for every column block nu
//    (p_j >> (L - l)) the sketch BO_nu = B(nu)^T O_l (R x C); for every pair of
//    slices of S^{l+1} that differ in i_{L-l} (bit l of k, merged row block
//    tau), the stacked sketch [V(2 tau, nu >> 1); V(2 tau + 1, nu >> 1)] BO_nu
//    (2r x C) is factored by QRCP; the halves of Q's first r columns are the
//    two slices and V(tau, nu) = Q^H [V(2 tau, .); V(2 tau + 1, .)].
//    Right levels l = 1 .. L - H mirror this for S^{L+2-l} with
//    AO_tau = A(tau)^T O'_l, the pair differing in j_{L-l} (bit 0 of k), and
//    the transposed halves of Q.
// 3. The slices of S^{H+1} (z1 when H = 0) are right-multiplied by
//    V(tau, nu) W(tau, nu)^T (Alg. 2's last line).
// The readings of the garbled middle-level indices are the pairwise stacking
// (the pairing of the App. A.3 orthogonalization) and H = floor(L / 2).
// QRCP: one warp per matrix; each step takes the remaining column of the
// largest residual norm (first on ties), orthogonalizes it twice against the
// columns already taken and normalizes it (so R has a real positive
// diagonal), then projects it out of the remaining columns.
#include <string>

#include "bfc_internal.h"

namespace bfc {

namespace {

__device__ __forceinline__ double2 dz() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double2 dmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) b
__device__ __forceinline__ double2 dcmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double2 wsum2(double2 v) { return make_double2(wsum(v.x), wsum(v.y)); }

// Column s of Q completed from the unit vector e_k whose residual
// 1 - sum_{i<s} |Q[k][i]|^2 against the columns taken is largest (first k on
// ties), orthogonalized twice and normalized; zero when no unit vector has a
// residual (Q already spans the rows).  Used past the numerical rank of M, so
// that Q keeps orthonormal columns there (as a Householder QR's Q does)
// instead of normalized rounding noise, which has no room left when M's rows
// span fewer dimensions than r (stacked coefficient blocks with zero rows).
__device__ void qr_complete(double2* Q, int rows, int r, int s, int lane)
{
    double bres = -1.0;
    int bk = rows;
    for (int k = lane; k < rows; k += 32) {
        double sq = 0.0;
        for (int i = 0; i < s; ++i) {
            const double2 v = Q[(size_t)k * r + i];
            sq += v.x * v.x + v.y * v.y;
        }
        const double res = 1.0 - sq;
        if (res > bres) {
            bres = res;
            bk = k;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ores = __shfl_xor_sync(0xffffffffu, bres, o);
        const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
        if (ores > bres || (ores == bres && ok < bk)) {
            bres = ores;
            bk = ok;
        }
    }
    if (!(bres > 1e-3) || bk >= rows) {
        for (int q = lane; q < rows; q += 32) Q[(size_t)q * r + s] = dz();
        __syncwarp();
        return;
    }
    // v = e_bk - Q (Q^H e_bk), then a second projection and the norm
    for (int q = lane; q < rows; q += 32) {
        double2 v = make_double2(q == bk ? 1.0 : 0.0, 0.0);
        for (int i = 0; i < s; ++i) {
            const double2 d = dmul(Q[(size_t)q * r + i], make_double2(Q[(size_t)bk * r + i].x, -Q[(size_t)bk * r + i].y));
            v.x -= d.x;
            v.y -= d.y;
        }
        Q[(size_t)q * r + s] = v;
    }
    __syncwarp();
    for (int i = 0; i < s; ++i) {
        double2 cf = dz();
        for (int q = lane; q < rows; q += 32) {
            const double2 d = dcmul(Q[(size_t)q * r + i], Q[(size_t)q * r + s]);
            cf.x += d.x;
            cf.y += d.y;
        }
        cf = wsum2(cf);
        __syncwarp();
        for (int q = lane; q < rows; q += 32) {
            const double2 d = dmul(cf, Q[(size_t)q * r + i]);
            Q[(size_t)q * r + s].x -= d.x;
            Q[(size_t)q * r + s].y -= d.y;
        }
        __syncwarp();
    }
    double nn = 0.0;
    for (int q = lane; q < rows; q += 32) {
        const double2 v = Q[(size_t)q * r + s];
        nn += v.x * v.x + v.y * v.y;
    }
    nn = wsum(nn);
    const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    for (int q = lane; q < rows; q += 32) {
        const double2 v = Q[(size_t)q * r + s];
        Q[(size_t)q * r + s] = make_double2(v.x * inv, v.y * inv);
    }
    __syncwarp();
}

// First r columns of Q of the column-pivoted QR of M (rows x C, row-major,
// overwritten by residuals) into Q (rows x r, row-major).  Past the numerical
// rank of M (a remaining column norm below 1e-13 of the largest initial one)
// the columns are orthonormal completions (qr_complete); past min(rows, r)
// they are zero.
__device__ void warp_qrcp(double2* M, int rows, int C, int r, double2* Q, int lane)
{
    uint32_t used = 0;
    double nmax0 = 0.0;
    for (int c = 0; c < C; ++c) {
        double nn = 0.0;
        for (int q = lane; q < rows; q += 32) {
            const double2 v = M[(size_t)q * C + c];
            nn += v.x * v.x + v.y * v.y;
        }
        nmax0 = fmax(nmax0, wsum(nn));
    }
    for (int s = 0; s < r; ++s) {
        int best = -1;
        double bestn = 0.0;
        if (s < rows && s < C) {
            for (int c = 0; c < C; ++c) {
                if (used >> c & 1u) continue;
                double nn = 0.0;
                for (int q = lane; q < rows; q += 32) {
                    const double2 v = M[(size_t)q * C + c];
                    nn += v.x * v.x + v.y * v.y;
                }
                nn = wsum(nn);
                if (nn > bestn) {
                    bestn = nn;
                    best = c;
                }
            }
        }
        if (best < 0 || !(bestn > 1e-26 * nmax0)) {
            if (s < rows) {
                qr_complete(Q, rows, r, s, lane);
            } else {
                for (int q = lane; q < rows; q += 32) Q[(size_t)q * r + s] = dz();
                __syncwarp();
            }
            continue;
        }
        used |= 1u << best;
        // the pivot column, orthogonalized twice against the columns taken
        for (int pass = 0; pass < 2; ++pass) {
            for (int i = 0; i < s; ++i) {
                double2 cf = dz();
                for (int q = lane; q < rows; q += 32) {
                    const double2 d = dcmul(Q[(size_t)q * r + i], M[(size_t)q * C + best]);
                    cf.x += d.x;
                    cf.y += d.y;
                }
                cf = wsum2(cf);
                __syncwarp();
                for (int q = lane; q < rows; q += 32) {
                    const double2 d = dmul(cf, Q[(size_t)q * r + i]);
                    M[(size_t)q * C + best].x -= d.x;
                    M[(size_t)q * C + best].y -= d.y;
                }
                __syncwarp();
            }
        }
        double nn = 0.0;
        for (int q = lane; q < rows; q += 32) {
            const double2 v = M[(size_t)q * C + best];
            nn += v.x * v.x + v.y * v.y;
        }
        nn = wsum(nn);
        const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
        for (int q = lane; q < rows; q += 32) {
            const double2 v = M[(size_t)q * C + best];
            Q[(size_t)q * r + s] = make_double2(v.x * inv, v.y * inv);
        }
        __syncwarp();
        // project the new direction out of the remaining columns
        for (int c = 0; c < C; ++c) {
            if (used >> c & 1u) continue;
            double2 cf = dz();
            for (int q = lane; q < rows; q += 32) {
                const double2 d = dcmul(Q[(size_t)q * r + s], M[(size_t)q * C + c]);
                cf.x += d.x;
                cf.y += d.y;
            }
            cf = wsum2(cf);
            __syncwarp();
            for (int q = lane; q < rows; q += 32) {
                const double2 d = dmul(cf, Q[(size_t)q * r + s]);
                M[(size_t)q * C + c].x -= d.x;
                M[(size_t)q * C + c].y -= d.y;
            }
            __syncwarp();
        }
    }
}

// out[blk][z][q] = sum_u X[blk * rows + u][z] O[(oglob ? blk * rows : 0) + u][q]
// (the transposed-times-Gaussian sketch of one block of rows); one thread per
// output element, rows summed in order.
__global__ void k_block_tn(const double2* __restrict__ X, int R, const double2* __restrict__ O, int C, int nblk,
                           int64_t rows, int oglob, double2* __restrict__ out)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nblk * R * C) return;
    const int blk = (int)(idx / ((int64_t)R * C));
    const int z = (int)((idx / C) % R), q = (int)(idx % C);
    const double2* Xb = X + (size_t)blk * rows * R;
    const double2* Ob = O + (oglob ? (size_t)blk * rows * C : 0);
    double2 acc = dz();
    for (int64_t u = 0; u < rows; ++u) {
        const double2 d = dmul(Xb[(size_t)u * R + z], Ob[(size_t)u * C + q]);
        acc.x += d.x;
        acc.y += d.y;
    }
    out[idx] = acc;
}

// Leaf blocks: M_tau = X(tau) XO (b x C), QRCP -> the block's factor rows
// (b x r) and coefficients Vout[tau] = Q^H X(tau) (r x R).  One warp per
// block; scratch of b (C + r) values per block.
__global__ void k_lr2bf_leaf(const double2* __restrict__ X, const double2* __restrict__ XO, int nblk, int b, int R,
                             int C, int r, double2* __restrict__ zout, double2* __restrict__ Vout,
                             double2* __restrict__ scratch)
{
    const int w = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= nblk) return;
    const double2* Xb = X + (size_t)w * b * R;
    double2* Ms = scratch + (size_t)w * b * (C + r);
    double2* Qs = Ms + (size_t)b * C;
    for (int x = lane; x < b * C; x += 32) {
        const int u = x / C, q = x % C;
        double2 acc = dz();
        for (int z = 0; z < R; ++z) {
            const double2 d = dmul(Xb[(size_t)u * R + z], XO[(size_t)z * C + q]);
            acc.x += d.x;
            acc.y += d.y;
        }
        Ms[x] = acc;
    }
    __syncwarp();
    warp_qrcp(Ms, b, C, r, Qs, lane);
    for (int x = lane; x < b * r; x += 32) zout[(size_t)w * b * r + x] = Qs[x];
    for (int a = 0; a < r; ++a)
        for (int z = 0; z < R; ++z) {
            double2 cf = dz();
            for (int u = lane; u < b; u += 32) {
                const double2 d = dcmul(Qs[(size_t)u * r + a], Xb[(size_t)u * R + z]);
                cf.x += d.x;
                cf.y += d.y;
            }
            cf = wsum2(cf);
            if (lane == 0) Vout[((size_t)w * r + a) * R + z] = cf;
        }
}

// One level of pairs.  Pair g gives its two halves and its new coefficients:
//   left  (side 0): tau = g / nnu, nu = g % nnu (nnu = 2^l); the two old
//         coefficient blocks are Vin[(2 tau + a) * 2^{l-1} + (nu >> 1)],
//         the sketch factor BO[nu]; halves into Z[l] at
//         k_a = ((2 tau + a) << l) | nu, as they are;
//   right (side 1): tau = g / nnu, nu = g % nnu (nnu = 2^{L-l}); old blocks
//         Vin[(tau >> 1) * 2^{L-l+1} + 2 nu + a], sketch factor AO[tau];
//         halves into Z[L+1-l] at k_a = (tau << (L+1-l)) | (2 nu + a),
//         transposed.
// Vout[g] = Q^H [old_0; old_1] (r x R).  One warp per pair; scratch of
// 2r (C + r) values per pair.
__global__ void k_lr2bf_pairs(const double2* __restrict__ Vin, const double2* __restrict__ SO, int side, int l, int L,
                              int R, int C, int r, int npairs, double2* __restrict__ Zlev,
                              double2* __restrict__ Vout, double2* __restrict__ scratch)
{
    const int g = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (g >= npairs) return;
    const int nnu = side == 0 ? (1 << l) : (1 << (L - l));
    const int tau = g / nnu, nu = g % nnu;
    const double2* old[2];
    const double2* F;
    if (side == 0) {
        for (int a = 0; a < 2; ++a) old[a] = Vin + ((size_t)(2 * tau + a) * (1 << (l - 1)) + (nu >> 1)) * r * R;
        F = SO + (size_t)nu * R * C;
    } else {
        for (int a = 0; a < 2; ++a) old[a] = Vin + ((size_t)(tau >> 1) * (1 << (L - l + 1)) + 2 * nu + a) * r * R;
        F = SO + (size_t)tau * R * C;
    }
    double2* Ms = scratch + (size_t)g * 2 * r * (C + r);
    double2* Qs = Ms + (size_t)2 * r * C;
    for (int x = lane; x < 2 * r * C; x += 32) {
        const int u = x / C, q = x % C;
        const double2* vr = old[u / r] + (size_t)(u % r) * R;
        double2 acc = dz();
        for (int z = 0; z < R; ++z) {
            const double2 d = dmul(vr[z], F[(size_t)z * C + q]);
            acc.x += d.x;
            acc.y += d.y;
        }
        Ms[x] = acc;
    }
    __syncwarp();
    warp_qrcp(Ms, 2 * r, C, r, Qs, lane);
    const int64_t S = (int64_t)1 << (L + 1);
    for (int a = 0; a < 2; ++a) {
        int64_t k;
        double2* Zs;
        if (side == 0) {
            k = ((int64_t)(2 * tau + a) << l) | nu;
            Zs = Zlev + (size_t)k * r * r;
            for (int x = lane; x < r * r; x += 32) Zs[x] = Qs[(size_t)(a * r + x / r) * r + x % r];
        } else {
            const int m = L + 1 - l;
            k = ((int64_t)tau << m) | (2 * nu + a);
            Zs = Zlev + (size_t)k * r * r;
            // slice (row c, column q) = Q half a, (row q, column c)
            for (int x = lane; x < r * r; x += 32) Zs[x] = Qs[(size_t)(a * r + x % r) * r + x / r];
        }
        (void)S;
    }
    for (int c = 0; c < r; ++c)
        for (int z = 0; z < R; ++z) {
            double2 cf = dz();
            for (int u = lane; u < 2 * r; u += 32) {
                const double2 d = dcmul(Qs[(size_t)u * r + c], old[u / r][(size_t)(u % r) * R + z]);
                cf.x += d.x;
                cf.y += d.y;
            }
            cf = wsum2(cf);
            if (lane == 0) Vout[((size_t)g * r + c) * R + z] = cf;
        }
}

// The middle step: T := T (V W^T) for every slice of S^{H+1} (H >= 1:
// block (tau, nu) = ((k >> H) >> 1, k mod 2^H), indexed tau 2^H + nu), or for
// the b rows z1 of every leaf block tau (H = 0).  One thread per target row.
__global__ void k_lr2bf_middle(double2* __restrict__ T, const double2* __restrict__ V, const double2* __restrict__ W,
                               int H, int64_t nrows_total, int rows_per_target, int R, int r)
{
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nrows_total) return;
    const int64_t tgt = row / rows_per_target;
    int64_t blk;
    if (H >= 1) {
        const int64_t tau = (tgt >> H) >> 1, nu = tgt & ((1 << H) - 1);
        blk = (tau << H) | nu;
    } else {
        blk = tgt;
    }
    const double2* Vb = V + (size_t)blk * r * R;
    const double2* Wb = W + (size_t)blk * r * R;
    double2 old[16];
    for (int a = 0; a < r; ++a) old[a] = T[(size_t)row * r + a];
    for (int c = 0; c < r; ++c) {
        double2 acc = dz();
        for (int a = 0; a < r; ++a) {
            double2 core = dz();   // (V W^T)[a][c]
            for (int z = 0; z < R; ++z) {
                const double2 d = dmul(Vb[(size_t)a * R + z], Wb[(size_t)c * R + z]);
                core.x += d.x;
                core.y += d.y;
            }
            const double2 d = dmul(old[a], core);
            acc.x += d.x;
            acc.y += d.y;
        }
        T[(size_t)row * r + c] = acc;
    }
}

}  // namespace

// Scratch layout (bytes) of lr2bf_run; see there.
size_t lr2bf_scratch_bytes(int64_t n, int L, int b, int R, int r, int p)
{
    const int C = r + p;
    const int64_t nb = (int64_t)1 << L;
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t so = up((size_t)nb * R * C * 16);                         // BO / AO per block
    const size_t vv = up((size_t)nb * r * R * 16);                         // one coefficient level
    const size_t leaf = (size_t)n * (C + r) * 16;
    const size_t pairs = (size_t)nb * 2 * r * (C + r) * 16;
    return so + 4 * vv + up(leaf > pairs ? leaf : pairs);
}

cudaError_t lr2bf_run(const double2* A, const double2* B, const double2* Gs, int64_t n, int L, int b, int R, int r,
                      int p, double2* z1, double2* Z, double2* zL, void* scratch, cudaStream_t st)
{
    const int C = r + p;
    const int H = L / 2, HR = L - H;
    const int64_t nb = (int64_t)1 << L;
    const int64_t S = (int64_t)1 << (L + 1);
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    char* base = (char*)scratch;
    double2* SO = (double2*)base;
    base += up((size_t)nb * R * C * 16);
    double2* Vb[2];
    double2* Wb[2];
    for (int q = 0; q < 2; ++q) {
        Vb[q] = (double2*)base;
        base += up((size_t)nb * r * R * 16);
    }
    for (int q = 0; q < 2; ++q) {
        Wb[q] = (double2*)base;
        base += up((size_t)nb * r * R * 16);
    }
    double2* work = (double2*)base;
    // Gaussian matrices: O_0 (n rows), left levels, right levels
    const double2* O0 = Gs;
    const double2* OL[32];
    const double2* OR[32];
    size_t off = (size_t)n * C;
    for (int l = 1; l <= H; ++l) {
        OL[l] = Gs + off;
        off += (size_t)(b << (L - l)) * C;
    }
    for (int l = 1; l <= HR; ++l) {
        OR[l] = Gs + off;
        off += (size_t)(b << (L - l)) * C;
    }
    const int nleaf = L == 0 ? 1 : (int)(n / b);
    const int lb = L == 0 ? (int)n : b;
    auto warps = [](int64_t w) { return (unsigned)((w * 32 + 127) / 128); };
    // 1. outer levels: z1, V and zL, W
    k_block_tn<<<(unsigned)((R * C + 127) / 128), 128, 0, st>>>(B, R, O0, C, 1, n, 1, SO);
    k_lr2bf_leaf<<<warps(nleaf), 128, 0, st>>>(A, SO, nleaf, lb, R, C, r, z1, Vb[0], work);
    k_block_tn<<<(unsigned)((R * C + 127) / 128), 128, 0, st>>>(A, R, O0, C, 1, n, 1, SO);
    k_lr2bf_leaf<<<warps(nleaf), 128, 0, st>>>(B, SO, nleaf, lb, R, C, r, zL, Wb[0], work);
    // 2. left levels
    int vc = 0;
    for (int l = 1; l <= H; ++l) {
        const int nnu = 1 << l;
        const int64_t rows = (int64_t)b << (L - l);
        k_block_tn<<<(unsigned)(((int64_t)nnu * R * C + 127) / 128), 128, 0, st>>>(B, R, OL[l], C, nnu, rows, 0, SO);
        k_lr2bf_pairs<<<warps(nb), 128, 0, st>>>(Vb[vc], SO, 0, l, L, R, C, r, (int)nb, Z + (size_t)(l - 1) * S * r * r,
                                                 Vb[vc ^ 1], work);
        vc ^= 1;
    }
    // right levels
    int wc = 0;
    for (int l = 1; l <= HR; ++l) {
        const int ntau = 1 << l;
        const int64_t rows = (int64_t)b << (L - l);
        const int m = L + 1 - l;
        k_block_tn<<<(unsigned)(((int64_t)ntau * R * C + 127) / 128), 128, 0, st>>>(A, R, OR[l], C, ntau, rows, 0, SO);
        k_lr2bf_pairs<<<warps(nb), 128, 0, st>>>(Wb[wc], SO, 1, l, L, R, C, r, (int)nb, Z + (size_t)(m - 1) * S * r * r,
                                                 Wb[wc ^ 1], work);
        wc ^= 1;
    }
    // 3. middle
    if (H >= 1) {
        const int64_t nrows = S * r;
        k_lr2bf_middle<<<(unsigned)((nrows + 127) / 128), 128, 0, st>>>(Z + (size_t)(H - 1) * S * r * r, Vb[vc],
                                                                       Wb[wc], H, nrows, r, R, r);
    } else {
        k_lr2bf_middle<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(z1, Vb[vc], Wb[wc], 0, n, lb, R, r);
    }
    return cudaGetLastError();
}

}  // namespace bfc
