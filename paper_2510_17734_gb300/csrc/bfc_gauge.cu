// Gauge fixing of the butterfly factors by left orthogonalization, in FP64
// on the master factors.  Eq. (BF_tensor_rep) is unchanged when an
// invertible r x r matrix G is inserted on a bond between two factors
// (X -> X G, Y -> G^{-1} Y).  Level by level, from S^1 to S^{L+1}, the
// matrix of every bond group is factored M = Q R (R with a real positive
// diagonal, so the factorization is unique) and replaced by Q, and R
// multiplies the factors on the other side of the bond:
//  * level 0, leaf block p of rows i: M = z1[p b .. p b + b - 1] (b x r),
//    R multiplies the slices 2p and 2p + 1 of S^2;
//  * level m = 1 .. L, bond (A, B) with k_{m+1} = ((A << 1 | a) << m) | B:
//    M = [Z[m][k(a = 0)]; Z[m][k(a = 1)]] (2r x r), R multiplies the slices
//    (A << (m + 1)) | (B << 1 | c), c = 0, 1, of S^{m+2} (m < L) or the
//    columns zL[j] of leaf block p_j = B (m = L).
// One warp per bond group, classical Gram-Schmidt applied twice per column
// (orthogonal to rounding level) with the rows spread over the lanes.
#include "bfc_internal.h"

namespace bfc {

namespace {

__device__ __forceinline__ double2 d2(double x, double y) { return make_double2(x, y); }

// Row q of the group's matrix (r complex values, contiguous).
struct GroupRows {
    double2* a;   // rows 0 .. split-1
    double2* b;   // rows split .. nrows-1
    int split, nrows, r;
    __device__ __forceinline__ double2* row(int q) const { return q < split ? a + (size_t)q * r : b + (size_t)(q - split) * r; }
};

template <int R>
__device__ void warp_qr(const GroupRows& M, double2 (*Rm)[R], int lane)
{
    for (int x = lane; x < R * R; x += 32) Rm[x / R][x % R] = d2(0.0, 0.0);
    __syncwarp();
    for (int j = 0; j < R; ++j) {
        for (int pass = 0; pass < 2; ++pass) {
            for (int i = 0; i < j; ++i) {
                double cx = 0.0, cy = 0.0;   // c = Q_i^H v
                for (int q = lane; q < M.nrows; q += 32) {
                    const double2 qi = M.row(q)[i], v = M.row(q)[j];
                    cx += qi.x * v.x + qi.y * v.y;
                    cy += qi.x * v.y - qi.y * v.x;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    cx += __shfl_xor_sync(0xffffffffu, cx, o);
                    cy += __shfl_xor_sync(0xffffffffu, cy, o);
                }
                __syncwarp();
                for (int q = lane; q < M.nrows; q += 32) {
                    double2* rw = M.row(q);
                    const double2 qi = rw[i];
                    double2 v = rw[j];
                    v.x -= cx * qi.x - cy * qi.y;
                    v.y -= cx * qi.y + cy * qi.x;
                    rw[j] = v;
                }
                if (lane == 0) {
                    Rm[i][j].x += cx;
                    Rm[i][j].y += cy;
                }
                __syncwarp();
            }
        }
        double s = 0.0;
        for (int q = lane; q < M.nrows; q += 32) {
            const double2 v = M.row(q)[j];
            s += v.x * v.x + v.y * v.y;
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const double nrm = sqrt(s);
        const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
        __syncwarp();
        for (int q = lane; q < M.nrows; q += 32) {
            double2* rw = M.row(q);
            rw[j].x *= inv;
            rw[j].y *= inv;
        }
        if (lane == 0) Rm[j][j] = d2(nrm, 0.0);
        __syncwarp();
    }
}

// T := Rm T for an r x r slice (row-major)
template <int R>
__device__ void left_mul_slice(double2* T, double2 (*Rm)[R], double2 (*tmp)[R], int lane)
{
    for (int x = lane; x < R * R; x += 32) tmp[x / R][x % R] = T[x];
    __syncwarp();
    for (int x = lane; x < R * R; x += 32) {
        const int a = x / R, c = x % R;
        double sx = 0.0, sy = 0.0;
        for (int k = a; k < R; ++k) {
            const double2 rk = Rm[a][k], t = tmp[k][c];
            sx += rk.x * t.x - rk.y * t.y;
            sy += rk.x * t.y + rk.y * t.x;
        }
        T[x] = d2(sx, sy);
    }
    __syncwarp();
}

template <int R>
__global__ void k_canon_level(double2* __restrict__ z1, double2* __restrict__ Z, double2* __restrict__ zL, int64_t n,
                              int L, int b, int level, int ngroups)
{
    __shared__ double2 Rs[4][R][R];
    __shared__ double2 Ts[4][R][R];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * 4 + w;
    if (g >= ngroups) return;
    const int64_t S = (int64_t)1 << (L + 1);
    auto slice = [&](int m, int64_t k) { return Z + ((size_t)(m - 1) * S + k) * R * R; };   // Z[m][k], m = 1..L
    GroupRows M;
    M.r = R;
    int A = 0, B = 0;
    if (level == 0) {
        M.a = z1 + (size_t)g * b * R;
        M.b = M.a;
        M.split = b;
        M.nrows = b;
    } else {
        A = g >> level;
        B = g & ((1 << level) - 1);
        M.a = slice(level, ((int64_t)(A << 1) << level) | B);
        M.b = slice(level, ((int64_t)(A << 1 | 1) << level) | B);
        M.split = R;
        M.nrows = 2 * R;
    }
    warp_qr<R>(M, Rs[w], lane);
    if (level == 0) {
        if (L >= 1) {
            left_mul_slice<R>(slice(1, 2 * (int64_t)g), Rs[w], Ts[w], lane);
            left_mul_slice<R>(slice(1, 2 * (int64_t)g + 1), Rs[w], Ts[w], lane);
        } else {
            // low-rank case (one bond over all rows): zL[j] := R zL[j]
            for (int64_t j = lane; j < n; j += 32) {
                double2 v[R];
#pragma unroll
                for (int c = 0; c < R; ++c) v[c] = zL[(size_t)j * R + c];
#pragma unroll
                for (int a = 0; a < R; ++a) {
                    double sx = 0.0, sy = 0.0;
                    for (int k = a; k < R; ++k) {
                        const double2 rk = Rs[w][a][k];
                        sx += rk.x * v[k].x - rk.y * v[k].y;
                        sy += rk.x * v[k].y + rk.y * v[k].x;
                    }
                    zL[(size_t)j * R + a] = d2(sx, sy);
                }
            }
        }
    } else if (level < L) {
        for (int c = 0; c < 2; ++c)
            left_mul_slice<R>(slice(level + 1, ((int64_t)A << (level + 1)) | (B << 1 | c)), Rs[w], Ts[w], lane);
    } else {
        for (int j = B * b + lane; j < (B + 1) * b; j += 32) {
            double2 v[R];
#pragma unroll
            for (int c = 0; c < R; ++c) v[c] = zL[(size_t)j * R + c];
#pragma unroll
            for (int a = 0; a < R; ++a) {
                double sx = 0.0, sy = 0.0;
                for (int k = a; k < R; ++k) {
                    const double2 rk = Rs[w][a][k];
                    sx += rk.x * v[k].x - rk.y * v[k].y;
                    sy += rk.x * v[k].y + rk.y * v[k].x;
                }
                zL[(size_t)j * R + a] = d2(sx, sy);
            }
        }
    }
}

// rows[q] := rows[q] X for `count` rows of r values (row vectors), X r x r
template <int R>
__device__ void right_mul_rows(double2* rows, int64_t count, const double2 (*X)[R], int lane)
{
    for (int64_t q = lane; q < count; q += 32) {
        double2 v[R];
#pragma unroll
        for (int c = 0; c < R; ++c) v[c] = rows[(size_t)q * R + c];
#pragma unroll
        for (int c = 0; c < R; ++c) {
            double sx = 0.0, sy = 0.0;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const double2 x = X[k][c];
                sx += v[k].x * x.x - v[k].y * x.y;
                sy += v[k].x * x.y + v[k].y * x.x;
            }
            rows[(size_t)q * R + c] = d2(sx, sy);
        }
    }
    __syncwarp();
}

// Right-to-left orthogonalization, one level (the mirror of k_canon_level):
//  * level L + 1, leaf block p of columns j: M = zL[p b .. p b + b - 1]
//    (b x r) = Q R, zL := Q and R^T right-multiplies the slices
//    (i_0 << L) | p of S^{L+1} (for L = 0: every row z1[i]);
//  * level m = L .. 1, group g: the two slices k = 2g, 2g + 1 of S^{m+1}
//    (differing in j_{m-1}, bit 0) form [Z0 | Z1] = R^H Q^H, computed as the
//    QR of the stacked conjugate transposes [Z0^H; Z1^H] (2r x r); Z_b :=
//    (half b of Q)^H, and R^H right-multiplies the two slices of S^m that
//    share the bond, ((g >> (m-1)) << m) | (c << (m-1)) | (g mod 2^(m-1)),
//    or, for m = 1, the rows z1[i] of leaf block p_i = g.
template <int R>
__global__ void k_rl_level(double2* __restrict__ z1, double2* __restrict__ Z, double2* __restrict__ zL, int64_t n,
                           int L, int b, int level, int ngroups)
{
    __shared__ double2 Rs[4][R][R];
    __shared__ double2 Xs[4][R][R];
    __shared__ double2 Ms[4][2 * R * R];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * 4 + w;
    if (g >= ngroups) return;
    const int64_t S = (int64_t)1 << (L + 1);
    auto slice = [&](int m, int64_t k) { return Z + ((size_t)(m - 1) * S + k) * R * R; };   // Z[m][k], m = 1..L
    GroupRows M;
    M.r = R;
    if (level == L + 1) {
        M.a = zL + (size_t)g * b * R;
        M.b = M.a;
        M.split = b;
        M.nrows = b;
        warp_qr<R>(M, Rs[w], lane);
        // X = R^T
        for (int x = lane; x < R * R; x += 32) Xs[w][x / R][x % R] = Rs[w][x % R][x / R];
        __syncwarp();
        if (L == 0) {
            right_mul_rows<R>(z1, n, Xs[w], lane);
        } else {
            for (int i0 = 0; i0 < 2; ++i0)
                right_mul_rows<R>(slice(L, ((int64_t)i0 << L) | g), R, Xs[w], lane);
        }
        return;
    }
    const int m = level;
    double2* Z0 = slice(m, 2 * (int64_t)g);
    double2* Z1 = slice(m, 2 * (int64_t)g + 1);
    // stacked conjugate transposes: row q < R is column q of Z0, conjugated
    for (int x = lane; x < 2 * R * R; x += 32) {
        const int q = x / R, a = x % R;
        const double2 v = q < R ? Z0[a * R + q] : Z1[a * R + (q - R)];
        Ms[w][x] = d2(v.x, -v.y);
    }
    __syncwarp();
    M.a = Ms[w];
    M.b = Ms[w];
    M.split = 2 * R;
    M.nrows = 2 * R;
    warp_qr<R>(M, Rs[w], lane);
    for (int x = lane; x < 2 * R * R; x += 32) {
        const int q = x / R, a = x % R;       // Q[q][a]
        const double2 v = Ms[w][x];
        if (q < R) Z0[a * R + q] = d2(v.x, -v.y);
        else Z1[a * R + (q - R)] = d2(v.x, -v.y);
    }
    // X = R^H
    for (int x = lane; x < R * R; x += 32) {
        const double2 v = Rs[w][x % R][x / R];
        Xs[w][x / R][x % R] = d2(v.x, -v.y);
    }
    __syncwarp();
    if (m > 1) {
        for (int c = 0; c < 2; ++c) {
            const int64_t kk = ((int64_t)(g >> (m - 1)) << m) | ((int64_t)c << (m - 1)) | (g & ((1 << (m - 1)) - 1));
            right_mul_rows<R>(slice(m - 1, kk), R, Xs[w], lane);
        }
    } else {
        right_mul_rows<R>(z1 + (size_t)g * b * R, b, Xs[w], lane);
    }
}

template <int R>
cudaError_t rl_all(double2* z1, double2* Z, double2* zL, int64_t n, int L, int b, cudaStream_t st)
{
    const int g0 = L == 0 ? 1 : (int)(n / b);
    k_rl_level<R><<<(g0 + 3) / 4, 128, 0, st>>>(z1, Z, zL, n, L, L == 0 ? (int)n : b, L + 1, g0);
    for (int m = L; m >= 1; --m) {
        const int g = 1 << L;
        k_rl_level<R><<<(g + 3) / 4, 128, 0, st>>>(z1, Z, zL, n, L, b, m, g);
    }
    return cudaGetLastError();
}

template <int R>
cudaError_t canon_one(double2* z1, double2* Z, double2* zL, int64_t n, int L, int b, int level, cudaStream_t st)
{
    if (level == 0) {
        const int g0 = L == 0 ? 1 : (int)(n / b);
        k_canon_level<R><<<(g0 + 3) / 4, 128, 0, st>>>(z1, Z, zL, n, L, L == 0 ? (int)n : b, 0, g0);
    } else {
        const int g = 1 << L;
        k_canon_level<R><<<(g + 3) / 4, 128, 0, st>>>(z1, Z, zL, n, L, b, level, g);
    }
    return cudaGetLastError();
}

template <int R>
cudaError_t canon_all(double2* z1, double2* Z, double2* zL, int64_t n, int L, int b, cudaStream_t st)
{
    const int g0 = L == 0 ? 1 : (int)(n / b);
    k_canon_level<R><<<(g0 + 3) / 4, 128, 0, st>>>(z1, Z, zL, n, L, L == 0 ? (int)n : b, 0, g0);
    for (int m = 1; m <= L; ++m) {
        const int g = 1 << L;
        k_canon_level<R><<<(g + 3) / 4, 128, 0, st>>>(z1, Z, zL, n, L, b, m, g);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_canonicalize(double2* z1, double2* Z, double2* zL, int64_t n, int L, int b, int r, cudaStream_t st)
{
    switch (r) {
    case 1: return canon_all<1>(z1, Z, zL, n, L, b, st);
    case 2: return canon_all<2>(z1, Z, zL, n, L, b, st);
    case 3: return canon_all<3>(z1, Z, zL, n, L, b, st);
    case 4: return canon_all<4>(z1, Z, zL, n, L, b, st);
    case 5: return canon_all<5>(z1, Z, zL, n, L, b, st);
    case 6: return canon_all<6>(z1, Z, zL, n, L, b, st);
    case 7: return canon_all<7>(z1, Z, zL, n, L, b, st);
    case 8: return canon_all<8>(z1, Z, zL, n, L, b, st);
    case 9: return canon_all<9>(z1, Z, zL, n, L, b, st);
    case 10: return canon_all<10>(z1, Z, zL, n, L, b, st);
    case 11: return canon_all<11>(z1, Z, zL, n, L, b, st);
    case 12: return canon_all<12>(z1, Z, zL, n, L, b, st);
    default: return cudaErrorInvalidValue;
    }
}

#define BFC_GAUGE_DISPATCH(FN, ...)                 \
    switch (r) {                                    \
    case 1: return FN<1>(__VA_ARGS__);              \
    case 2: return FN<2>(__VA_ARGS__);              \
    case 3: return FN<3>(__VA_ARGS__);              \
    case 4: return FN<4>(__VA_ARGS__);              \
    case 5: return FN<5>(__VA_ARGS__);              \
    case 6: return FN<6>(__VA_ARGS__);              \
    case 7: return FN<7>(__VA_ARGS__);              \
    case 8: return FN<8>(__VA_ARGS__);              \
    case 9: return FN<9>(__VA_ARGS__);              \
    case 10: return FN<10>(__VA_ARGS__);            \
    case 11: return FN<11>(__VA_ARGS__);            \
    case 12: return FN<12>(__VA_ARGS__);            \
    default: return cudaErrorInvalidValue;          \
    }

cudaError_t launch_canon_level(double2* z1, double2* Z, double2* zL, int64_t n, int L, int b, int r, int level,
                               cudaStream_t st)
{
    BFC_GAUGE_DISPATCH(canon_one, z1, Z, zL, n, L, b, level, st)
}

cudaError_t launch_rl_orthogonalize(double2* z1, double2* Z, double2* zL, int64_t n, int L, int b, int r,
                                    cudaStream_t st)
{
    BFC_GAUGE_DISPATCH(rl_all, z1, Z, zL, n, L, b, st)
}

}  // namespace bfc
