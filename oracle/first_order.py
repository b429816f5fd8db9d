"""First-order butterfly completion and the orthogonalization sweeps (float64
/ complex128 oracle, numpy; test infrastructure, shares no code with the
CUDA library).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.

Functions and the passage each follows:
  envs                  left / right environments of every observed entry
                        (the vectors u and v of Alg. 1 and Alg. 4)
  adam_iteration        Alg. 4 (ADAM for butterfly completion) with the
                        update of Alg. 3
  lr_orthogonalize      the right-to-left orthogonalization sweep of App. A.3
                        (LQ of the slice pairs, the triangle absorbed into
                        the left neighbour)
  adf_iteration         Alg. 5 (ADF for butterfly completion) with the
                        left-to-right QR and absorb steps of App. A.3

Packed factors are [z1 (n r) | Z (L 2^{L+1} r^2) | zL (n r)] complex128,
x_ij = z1[i]^T Z[1][k_2] ... Z[L][k_{L+1}] zL[j], with the slice id
k_{m+1} = ((p_i >> (m-1)) << m) | (p_j >> (L-m)), p = index // b (Eq.
(indices), App. A.2).

Readings (listed with the other readings of the paper in the design notes):
* complex parameters are treated as (Re, Im) pairs of reals; the gradient
  of f = 1/2 sum |x - t|^2 + lambda/2 ||S||^2 is packed df/dRe + i df/dIm
  = sum (x - t) conj(a) + lambda s, and ADAM's moments run on the two reals
  separately (g * g is the square of each real);
* Alg. 4 updates one factor at a time (l = 1 .. L+2), each gradient taken
  with the newest values of all other factors; the bias correction uses the
  outer iteration t;
* ADF (Alg. 5): the direction of slice s is the negative gradient
  N_s = sum_{e in s} G_e conj(a_e) - lambda S_s with G = t - x; the step is
  the exact minimizer of f along it,
  alpha_s = ||N_s||^2 / (||z_s||^2 + lambda ||N_s||^2), z_e = a_e . N_s
  (with lambda = 0 this is the printed ||N_s||^2 / ||z||^2);
  S_s += alpha_s N_s, G_e -= alpha_s z_e; after the update of factor l
  (l <= L+1) its bond groups are QR-factored and R moves into factor l+1;
  the right-to-left sweep that makes the factors right of the centre
  orthonormal runs at the start of every iteration (printed once before the
  loop);
* every QR is made unique by a real positive diagonal of R.
"""
from __future__ import annotations

import numpy as np


def split(X, n, L, r):
    S = 1 << (L + 1)
    z1 = X[:n * r].reshape(n, r)
    Z = X[n * r:n * r + L * S * r * r].reshape(L, S, r, r)
    zL = X[n * r + L * S * r * r:].reshape(n, r)
    return z1, Z, zL


def slice_keys(i, j, L, b):
    """k_{m+1} for m = 1..L (list index m - 1)."""
    pi, pj = np.asarray(i, np.int64) // b, np.asarray(j, np.int64) // b
    return [((pi >> (m - 1)) << m) | (pj >> (L - m)) for m in range(1, L + 1)]


def right_envs(z1, Z, zL, i, j, L, keys):
    """w_m for m = L..0: w_L = zL[j], w_{m-1} = Z[m][k_{m+1}] w_m."""
    w = [None] * (L + 1)
    w[L] = zL[j]
    for m in range(L, 0, -1):
        w[m - 1] = np.einsum("eac,ec->ea", Z[m - 1][keys[m - 1]], w[m])
    return w


def envs(n, L, b, r, X, i, j):
    """(h, w): h[m] (m = 1..L+1) left, w[m] (m = 0..L) right environments,
    so that x = h_m^T Z[m][k_{m+1}] w_m for every m."""
    z1, Z, zL = split(np.asarray(X, np.complex128), n, L, r)
    keys = slice_keys(i, j, L, b)
    w = right_envs(z1, Z, zL, i, j, L, keys)
    h = {1: z1[i]}
    for m in range(1, L + 1):
        h[m + 1] = np.einsum("ea,eac->ec", h[m], Z[m - 1][keys[m - 1]])
    return h, w


def _segment_sum(idx, vals, K):
    out = np.zeros((K,) + vals.shape[1:], dtype=vals.dtype)
    np.add.at(out, idx, vals)
    return out


# ------------------------------------------------------------------- ADAM

def adam_update(s, g, M, V, alpha, beta1, beta2, sigma, t):
    """Alg. 3 on the real and imaginary parts of complex arrays s, g (M, V
    real arrays of shape s.shape + (2,)); returns the new s (M, V in place)."""
    gr = np.stack([g.real, g.imag], axis=-1)
    M *= beta1
    M += (1.0 - beta1) * gr
    V *= beta2
    V += (1.0 - beta2) * gr * gr
    mh = M / (1.0 - beta1 ** t)
    vh = V / (1.0 - beta2 ** t)
    step = alpha * mh / (np.sqrt(vh) + sigma)
    return s - (step[..., 0] + 1j * step[..., 1])


def adam_iteration(n, L, b, r, lam, X, i, j, t, M, V, it, alpha=1e-3, beta1=0.9, beta2=0.999,
                   sigma=1e-8):
    """One outer iteration (number it >= 1) of Alg. 4: for S^1, S^2 ..
    S^{L+1}, S^{L+2} in turn, the gradient of f with respect to that factor
    at the newest values of all factors, then the Alg. 3 update of that
    factor.  M, V: real arrays of shape (P, 2) (moments of the packed
    parameters), updated in place.  Returns the new packed factors."""
    X = np.asarray(X, np.complex128).copy()
    z1, Z, zL = split(X, n, L, r)
    Mz1, MZ, MzL = split_moments(M, n, L, r)
    Vz1, VZ, VzL = split_moments(V, n, L, r)
    i = np.asarray(i)
    j = np.asarray(j)
    t = np.asarray(t, np.complex128)
    keys = slice_keys(i, j, L, b)
    w = right_envs(z1, Z, zL, i, j, L, keys)
    # S^1: design w_0
    x = np.einsum("ea,ea->e", z1[i], w[0])
    G = _segment_sum(i, (x - t)[:, None] * np.conj(w[0]), n) + lam * z1
    z1[:] = adam_update(z1, G, Mz1, Vz1, alpha, beta1, beta2, sigma, it)
    h = z1[i]
    for m in range(1, L + 1):
        k = keys[m - 1]
        Zm = Z[m - 1]
        x = np.einsum("ea,eac,ec->e", h, Zm[k], w[m])
        a = np.einsum("ea,ec->eac", h, w[m])
        G = _segment_sum(k, (x - t)[:, None, None] * np.conj(a), Zm.shape[0]) + lam * Zm
        Zm[:] = adam_update(Zm, G, MZ[m - 1], VZ[m - 1], alpha, beta1, beta2, sigma, it)
        h = np.einsum("ea,eac->ec", h, Zm[k])
    x = np.einsum("ec,ec->e", h, zL[j])
    G = _segment_sum(j, (x - t)[:, None] * np.conj(h), n) + lam * zL
    zL[:] = adam_update(zL, G, MzL, VzL, alpha, beta1, beta2, sigma, it)
    return X


def split_moments(M, n, L, r):
    S = 1 << (L + 1)
    a = n * r
    z = L * S * r * r
    return (M[:a].reshape(n, r, 2), M[a:a + z].reshape(L, S, r, r, 2), M[a + z:].reshape(n, r, 2))


# --------------------------------------------------------- orthogonalization

def qr_pos(M):
    """Reduced QR with a real non-negative diagonal of R (unique when M has
    full column rank)."""
    Q, Rm = np.linalg.qr(M)
    d = np.diag(Rm).copy()
    ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1.0), 1.0)
    return Q * ph[None, :], np.conj(ph)[:, None] * Rm


def lr_orthogonalize(n, L, b, r, X):
    """Right-to-left orthogonalization sweep (App. A.3, mirrored): the leaf
    blocks of zL (b x r, rows j of one prefix p_j) become Q of their QR and
    the slices Z[L][(i_0 << L) | p_j] take R^T on the right; for m = L .. 1
    the two slices of Z[m] that differ in j_{m-1} (bit 0 of k_{m+1}) form
    [Z0 | Z1] = R^H Q^H (the LQ factorization, by QR of its conjugate
    transpose), become the two halves of Q^H, and R^H moves right-multiplied
    into the slices of the left neighbour that share the bond (the pair of
    Z[m-1] differing in i_{L-m+1}, bit m-1 of k_m; the rows z1[i] of the
    leaf block p_i for m = 1).  Entries are unchanged; every factor but z1
    ends right-orthonormal.  Needs b >= r."""
    X = np.asarray(X, np.complex128).copy()
    z1, Z, zL = split(X, n, L, r)
    if L == 0:
        Q, Rm = qr_pos(zL)
        zL[:] = Q
        z1[:] = z1 @ Rm.T
        return X
    for p in range(n // b):
        rows = slice(p * b, (p + 1) * b)
        Q, Rm = qr_pos(zL[rows])
        zL[rows] = Q
        for i0 in (0, 1):
            k = (i0 << L) | p
            Z[L - 1, k] = Z[L - 1, k] @ Rm.T
    for m in range(L, 0, -1):
        for g in range(1 << L):
            k0, k1 = g << 1, (g << 1) | 1
            Mh = np.hstack([Z[m - 1, k0], Z[m - 1, k1]]).conj().T      # 2r x r
            Q, Rm = qr_pos(Mh)
            Z[m - 1, k0] = Q[:r].conj().T
            Z[m - 1, k1] = Q[r:].conj().T
            Rh = Rm.conj().T
            if m > 1:
                for bit in (0, 1):
                    kk = ((g >> (m - 1)) << m) | (bit << (m - 1)) | (g & ((1 << (m - 1)) - 1))
                    Z[m - 2, kk] = Z[m - 2, kk] @ Rh
            else:
                rows = slice(g * b, (g + 1) * b)
                z1[rows] = z1[rows] @ Rh
    return X


def _qr_absorb_level(n, L, b, r, z1, Z, zL, level):
    """Left-to-right QR of one factor (App. A.3): level 0 = the leaf blocks of
    z1 (R into the pair of Z[1] slices the block reaches), level m = 1..L =
    the slice pairs of Z[m] differing in i_{L-m} (bit m), stacked 2r x r (R
    into the two slices of Z[m+1] that share the bond, or the leaf block of
    zL when m = L)."""
    if level == 0:
        if L == 0:
            Q, Rm = qr_pos(z1)
            z1[:] = Q
            zL[:] = (Rm @ zL.T).T
            return
        for p in range(n // b):
            rows = slice(p * b, (p + 1) * b)
            Q, Rm = qr_pos(z1[rows])
            z1[rows] = Q
            for a in (0, 1):
                Z[0, 2 * p + a] = Rm @ Z[0, 2 * p + a]
        return
    m = level
    for A in range(1 << (L - m)):
        for B in range(1 << m):
            k0 = ((A << 1) << m) | B
            k1 = (((A << 1) | 1) << m) | B
            Q, Rm = qr_pos(np.vstack([Z[m - 1, k0], Z[m - 1, k1]]))
            Z[m - 1, k0] = Q[:r]
            Z[m - 1, k1] = Q[r:]
            if m < L:
                for c in (0, 1):
                    kk = (A << (m + 1)) | (B << 1) | c
                    Z[m, kk] = Rm @ Z[m, kk]
            else:
                rows = slice(B * b, (B + 1) * b)
                zL[rows] = (Rm @ zL[rows].T).T


# -------------------------------------------------------------------- ADF

def _adf_block_step(keys, K, a_flat, G, S_flat, lam):
    """Slice-wise steepest descent with exact line search: returns the new
    slices and the new residual."""
    N = _segment_sum(keys, G[:, None] * np.conj(a_flat), K) - lam * S_flat
    z = np.einsum("ed,ed->e", a_flat, N[keys])
    nn = np.sum(np.abs(N) ** 2, axis=1)
    zz = _segment_sum(keys, np.abs(z) ** 2, K)
    den = zz + lam * nn
    alpha = np.where(den > 0, nn / np.where(den > 0, den, 1.0), 0.0)
    return S_flat + alpha[:, None] * N, G - alpha[keys] * z


def adf_iteration(n, L, b, r, lam, X, i, j, t, trace=None):
    """One iteration of Alg. 5: right-to-left orthogonalization, residual
    G = t - x, then for each factor in turn (S^1, S^2 .. S^{L+1}, S^{L+2})
    the slice-wise exact-line-search step along the negative gradient and
    (except for S^{L+2}) the QR of its bond groups with R absorbed into the
    next factor.  Returns (new packed factors, ||G|| / ||t||).  `trace` (a
    list) receives (level, factors before, factors after) of every factor
    update, for the tests."""
    X = lr_orthogonalize(n, L, b, r, X)
    z1, Z, zL = split(X, n, L, r)
    i = np.asarray(i)
    j = np.asarray(j)
    t = np.asarray(t, np.complex128)
    keys = slice_keys(i, j, L, b)
    w = right_envs(z1, Z, zL, i, j, L, keys)
    G = t - np.einsum("ea,ea->e", z1[i], w[0])
    before = X.copy() if trace is not None else None
    new, G = _adf_block_step(i, n, w[0], G, z1, lam)
    z1[:] = new
    if trace is not None:
        trace.append((0, before, X.copy()))
    _qr_absorb_level(n, L, b, r, z1, Z, zL, 0)
    h = z1[i]
    for m in range(1, L + 1):
        k = keys[m - 1]
        a = np.einsum("ea,ec->eac", h, w[m]).reshape(len(k), r * r)
        Zm = Z[m - 1]
        before = X.copy() if trace is not None else None
        new, G = _adf_block_step(k, Zm.shape[0], a, G, Zm.reshape(-1, r * r), lam)
        Zm[:] = new.reshape(Zm.shape)
        if trace is not None:
            trace.append((m, before, X.copy()))
        _qr_absorb_level(n, L, b, r, z1, Z, zL, m)
        h = np.einsum("ea,eac->ec", h, Zm[k])
    before = X.copy() if trace is not None else None
    new, G = _adf_block_step(j, n, h, G, zL, lam)
    zL[:] = new
    if trace is not None:
        trace.append((L + 1, before, X.copy()))
    return X, float(np.linalg.norm(G) / np.linalg.norm(t))
