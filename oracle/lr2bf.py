"""Randomized low-rank to butterfly conversion (Alg. 2 of the paper, Sec.
4.2), float64 / complex128 oracle in numpy; test infrastructure that shares
no code with the CUDA library.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.

Input: X = A B^T (A, B: n x R), levels L, leaf size b (n = b 2^L), rank r,
oversampling p, and the Gaussian sketch matrices (passed in; see
gaussian_layout).  Output: packed butterfly factors [z1 | Z | zL].

Notation: p_i = i // b; at left level l the row blocks are tau = p_i >> l
(the L - l leading bits i_0 .. i_{L-l-1}) and the column blocks
nu = p_j >> (L - l) (j_0 .. j_{l-1}); at right level l the row blocks are
p_i >> (L - l) and the column blocks p_j >> l.

Steps (the paper's order; readings of its garbled indices in brackets):
1. Outer sketches M = A (B^T O_0) and N = B (A^T O_0) (n x (r + p)).
   For every leaf block, QR with column pivoting of its b rows of M
   (resp. N): the first r columns of Q are the rows z1[i] (resp. zL[j]) of
   the block, and V = Q_r^H A(block, :) (resp. W = Q_r^H B(block, :)),
   r x R, the block's coefficients in the new basis.
2. Left levels l = 1 .. H, H = floor(L / 2): for every slice k of S^{l+1}
   (row block tau' = p_i >> (l-1), column block nu = p_j >> (L-l)) the
   sketch M(k) = V(tau', nu >> 1) B(nu, :)^T O_l (r x (r + p)), O_l a
   Gaussian over the b 2^{L-l} columns of nu.  [The two slices that differ
   in i_{L-l} (bit l of k) share the merged row block tau' >> 1: their
   sketches are stacked (2r x (r + p)) and factored together by QRCP; the
   first r columns of Q, split in halves, are the two slices, and
   V(tau' >> 1, nu) = Q_r^H [V(tau'_0, nu >> 1); V(tau'_1, nu >> 1)].  The
   orthogonalization sweeps of App. A.3 pair the slices over the same bit.]
   Right levels l = 1 .. L - H mirror this for S^{L+2-l} with
   N(k) = W(tau >> 1, nu') A(tau, :)^T O'_l, the pair differing in j_{L-l}
   (bit 0 of k), and S^{L+2-l}(k_b) = (half b of Q_r)^T.
3. The middle: the slices of S^{H+1} (the last left level; z1 when H = 0)
   are right-multiplied by V(tau, nu) W(tau, nu)^T (Alg. 2's last line),
   the two coefficient matrices of the block they close.
With R <= r and leaf blocks of full column rank this reproduces A B^T to
rounding.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def num_levels(L):
    """(left, right) levels of Alg. 2: H = floor(L / 2) and L - H."""
    return L // 2, L - L // 2


def gaussian_layout(n, L, b, r, p):
    """Row counts of the sketch matrices, in the order they are packed:
    O_0 (n rows), then O_l for the left levels l = 1 .. H, then O'_l for the
    right levels l = 1 .. L - H (b 2^{L-l} rows each); every matrix has
    r + p complex columns, row-major."""
    H, HR = num_levels(L)
    rows = [n] + [b << (L - l) for l in range(1, H + 1)] + [b << (L - l) for l in range(1, HR + 1)]
    return rows, r + p


def _unpack_gaussians(G, n, L, b, r, p):
    rows, cols = gaussian_layout(n, L, b, r, p)
    G = np.asarray(G, np.complex128).ravel()
    assert G.size == sum(rows) * cols, (G.size, sum(rows) * cols)
    out, off = [], 0
    for nr in rows:
        out.append(G[off:off + nr * cols].reshape(nr, cols))
        off += nr * cols
    H, HR = num_levels(L)
    return out[0], out[1:1 + H], out[1 + H:]


def qrcp_basis(M, r):
    """First r columns of Q of the column-pivoted QR of M (LAPACK geqp3),
    each column's phase fixed so that the diagonal of R is real and
    non-negative; zero columns when M has fewer than r rows."""
    Q, Rm, _ = sla.qr(M, mode="economic", pivoting=True)
    d = np.diag(Rm)
    ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1.0), 1.0)
    Q = Q * ph[None, :]
    out = np.zeros((M.shape[0], r), dtype=np.complex128)
    c = min(r, Q.shape[1])
    out[:, :c] = Q[:, :c]
    return out


def lr_to_butterfly(n, L, b, r, A, B, gaussians, p):
    """Alg. 2: butterfly factors (packed complex128) of X = A B^T."""
    A = np.asarray(A, np.complex128)
    B = np.asarray(B, np.complex128)
    O0, OL, OR = _unpack_gaussians(gaussians, n, L, b, r, p)
    H, HR = num_levels(L)
    S = 1 << (L + 1)
    z1 = np.zeros((n, r), np.complex128)
    zL = np.zeros((n, r), np.complex128)
    Z = np.zeros((L, S, r, r), np.complex128)
    nblk = n // b
    # 1. outer levels
    M = A @ (B.T @ O0)
    N = B @ (A.T @ O0)
    V = {}
    W = {}
    for q in range(nblk):
        rows = slice(q * b, (q + 1) * b)
        Q = qrcp_basis(M[rows], r)
        z1[rows] = Q
        V[(q, 0)] = Q.conj().T @ A[rows]
        Q = qrcp_basis(N[rows], r)
        zL[rows] = Q
        W[(0, q)] = Q.conj().T @ B[rows]
    # 2. left levels: V is keyed by (row block, column block) of the level
    for l in range(1, H + 1):
        Vn = {}
        ncol = b << (L - l)
        for tau in range(1 << (L - l)):
            for nu in range(1 << l):
                Bnu = B[nu * ncol:(nu + 1) * ncol]
                BO = Bnu.T @ OL[l - 1]                       # R x (r + p)
                V0, V1 = V[(2 * tau, nu >> 1)], V[(2 * tau + 1, nu >> 1)]
                Msk = np.vstack([V0 @ BO, V1 @ BO])          # 2r x (r + p)
                Q = qrcp_basis(Msk, r)
                k0 = ((2 * tau) << l) | nu
                k1 = ((2 * tau + 1) << l) | nu
                Z[l - 1, k0] = Q[:r]
                Z[l - 1, k1] = Q[r:]
                Vn[(tau, nu)] = Q.conj().T @ np.vstack([V0, V1])
        V = Vn
    # right levels: W keyed by (row block, column block) of the level
    for l in range(1, HR + 1):
        m = L + 1 - l
        Wn = {}
        nrow = b << (L - l)
        for tau in range(1 << l):
            Atau = A[tau * nrow:(tau + 1) * nrow]
            AO = Atau.T @ OR[l - 1]
            for nu in range(1 << (L - l)):
                W0, W1 = W[(tau >> 1, 2 * nu)], W[(tau >> 1, 2 * nu + 1)]
                Nsk = np.vstack([W0 @ AO, W1 @ AO])
                Q = qrcp_basis(Nsk, r)
                k0 = (tau << m) | (2 * nu)
                k1 = (tau << m) | (2 * nu + 1)
                Z[m - 1, k0] = Q[:r].T
                Z[m - 1, k1] = Q[r:].T
                Wn[(tau, nu)] = Q.conj().T @ np.vstack([W0, W1])
        W = Wn
    # 3. middle: the core V W^T of every block closes the last left level
    if H == 0:
        for tau in range(nblk):
            C = V[(tau, 0)] @ W[(tau, 0)].T
            rows = slice(tau * b, (tau + 1) * b)
            z1[rows] = z1[rows] @ C
    else:
        for k in range(S):
            tau = (k >> H) >> 1
            nu = k & ((1 << H) - 1)
            Z[H - 1, k] = Z[H - 1, k] @ (V[(tau, nu)] @ W[(tau, nu)].T)
    return np.concatenate([z1.ravel(), Z.ravel(), zL.ravel()])
