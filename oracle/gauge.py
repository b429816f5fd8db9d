"""Gauge fixing of butterfly factors by left orthogonalization (float64
oracle, test infrastructure; shares no code with the CUDA library).

The entry formula x_ij = z1[i] Z[1][k_2] ... Z[L][k_{L+1}] zL[j]
(Eq. (BF_tensor_rep)) is unchanged when an invertible r x r matrix G is
inserted on a bond, X -> X G and Y -> G^{-1} Y for the two factors the bond
joins (the gauge freedom of a tensor network, Sec. 2).  Left
orthogonalization removes it level by level:

* level 0: the rows z1[i] of one leaf block p (i = p b .. p b + b - 1) form
  a b x r matrix M = Q R; they become the rows of Q and R multiplies the two
  slices of S^2 that the block reaches, Z[1][2p] and Z[1][2p + 1];
* level m = 1 .. L: with k_{m+1} = ((A << 1 | a) << m) | B (A the high
  bits of p_i, a the next bit, B the m high bits of p_j), the two slices
  a = 0, 1 of a bond (A, B) are stacked into a 2r x r matrix = Q R; they
  become the two halves of Q and R multiplies the factors on the other side
  of the bond: the two slices c = 0, 1 of S^{m+2},
  k_{m+2} = (A << (m + 1)) | (B << 1 | c), for m < L, and the columns zL[j]
  of the leaf block p_j = B for m = L.

Each QR is made unique by a real positive diagonal of R.  The result is the
same tensor with every factor but zL left-orthonormal; zL carries the norm.
"""
from __future__ import annotations

import numpy as np


def _qr_pos(M):
    Q, Rm = np.linalg.qr(M)
    d = np.diag(Rm).copy()
    ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1.0), 1.0)
    return Q * ph[None, :], np.conj(ph)[:, None] * Rm


def canonicalize(n, L, b, r, packed):
    """Left-orthogonal gauge of packed factors [z1 | Z | zL] (complex128)."""
    X = np.asarray(packed, dtype=np.complex128).copy()
    S = 1 << (L + 1)
    z1 = X[:n * r].reshape(n, r)
    Z = X[n * r:n * r + L * S * r * r].reshape(L, S, r, r) if L > 0 else None
    zL = X[n * r + L * S * r * r:].reshape(n, r)
    nblk = n // b
    if L == 0:
        # low-rank case: x = z1[i] . zL[j]; one bond over all rows
        Q, Rm = _qr_pos(z1)
        z1[:] = Q
        zL[:] = (Rm @ zL.T).T
        return X
    for p in range(nblk):
        Q, Rm = _qr_pos(z1[p * b:(p + 1) * b])
        z1[p * b:(p + 1) * b] = Q
        for a in (0, 1):
            Z[0, 2 * p + a] = Rm @ Z[0, 2 * p + a]
    for m in range(1, L + 1):
        for A in range(1 << (L - m)):
            for B in range(1 << m):
                k0 = ((A << 1 | 0) << m) | B
                k1 = ((A << 1 | 1) << m) | B
                M = np.vstack([Z[m - 1, k0], Z[m - 1, k1]])
                Q, Rm = _qr_pos(M)
                Z[m - 1, k0] = Q[:r]
                Z[m - 1, k1] = Q[r:]
                if m < L:
                    for c in (0, 1):
                        kk = (A << (m + 1)) | (B << 1 | c)
                        Z[m, kk] = Rm @ Z[m, kk]
                else:
                    rows = slice(B * b, (B + 1) * b)
                    zL[rows] = (Rm @ zL[rows].T).T
    return X
