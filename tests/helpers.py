"""Test-side helpers: the test's own reading of the packed factor layout
(numpy reshapes of the App. A.2 reshape) and tolerance measures.  Shared by
the oracle pins and the GPU parity tests; independent of both the oracle's C
code and the CUDA library."""
import math

import numpy as np


def split_packed(packed, n, L, b, r):
    S = 1 << (L + 1)
    z1 = packed[: n * r].reshape(n, r)
    Z = packed[n * r: n * r + L * S * r * r].reshape(L, S, r, r)
    zL = packed[n * r + L * S * r * r:].reshape(n, r)
    return z1, Z, zL


def join_packed(z1, Z, zL):
    return np.concatenate([z1.ravel(), Z.ravel(), zL.ravel()])


def level_keys(i, j, L, b):
    """Slice keys of the middle factors, keys[m-1] for S^{m+1}."""
    pi, pj = np.asarray(i) // b, np.asarray(j) // b
    return [((pi >> (m - 1)) << m) | (pj >> (L - m)) for m in range(1, L + 1)]


def envs_numpy(z1, Z, zL, i, j, L, b, r):
    """Left envs h_m (m = 1..L+1) and right envs w_m (m = 0..L) per entry."""
    pi, pj = np.asarray(i) // b, np.asarray(j) // b
    Zt = [Z[m].reshape((2,) * (L + 1) + (r, r)) for m in range(L)]
    ib = [(pi >> (L - 1 - q)) & 1 for q in range(L)]
    jb = [(pj >> (L - 1 - q)) & 1 for q in range(L)]

    def slice_mats(m):
        return Zt[m - 1][tuple(ib[: L - m + 1]) + tuple(jb[:m])]

    h = {1: z1[i]}
    for m in range(1, L + 1):
        h[m + 1] = np.einsum("ea,eac->ec", h[m], slice_mats(m))
    w = {L: zL[j]}
    for m in range(L, 0, -1):
        w[m - 1] = np.einsum("eac,ec->ea", slice_mats(m), w[m])
    return h, w


def lstsq_block(A, t, lam):
    d = A.shape[1]
    Aa = np.vstack([A, math.sqrt(lam) * np.eye(d)])
    ta = np.concatenate([t, np.zeros(d)])
    return np.linalg.lstsq(Aa, ta, rcond=None)[0]


def block_objective(A, t, lam, s):
    res = A @ s - t
    return float(np.vdot(res, res).real + lam * np.vdot(s, s).real)


def rel_dev(x, ref):
    """Max over entries of |x - ref| / max(|ref|, rms(ref))."""
    x, ref = np.asarray(x), np.asarray(ref)
    rms = math.sqrt(float(np.mean(np.abs(ref) ** 2))) if ref.size else 1.0
    den = np.maximum(np.abs(ref), rms if rms > 0 else 1.0)
    return float(np.max(np.abs(x - ref) / den)) if ref.size else 0.0


def block_conditions(X0, X1, i, j, t, n, L, b, r, lam, ridge_rel=0.0):
    """Condition numbers of every block system K + lambda_eff I of one ALS
    sweep from X0 that produced X1 (Alg. 1 order: each level's design from the
    new factors left of it and the old factors right of it), with
    lambda_eff = max(lam, ridge_rel trace(K) / dim).  Returns a list with one
    array of condition numbers per level (S^1, the middle factors, S^{L+2})."""
    z1o, Zo, zLo = split_packed(X0, n, L, b, r)
    z1n, Zn, zLn = split_packed(X1, n, L, b, r)
    i, j = np.asarray(i), np.asarray(j)

    def cond(A):
        K = A.conj().T @ A
        d = K.shape[0]
        le = max(lam, ridge_rel * float(np.trace(K).real) / d)
        ev = np.linalg.eigvalsh(K + le * np.eye(d))
        return float(ev[-1] / ev[0]) if ev[0] > 0 else float("inf")

    out = []
    _, w_old = envs_numpy(z1o, Zo, zLo, i, j, L, b, r)
    out.append(np.array([cond(w_old[0][i == row]) for row in range(n) if np.any(i == row)]))
    pi, pj = i // b, j // b
    for m in range(1, L + 1):
        Zmix = np.concatenate([Zn[: m - 1], Zo[m - 1:]])
        h_new, _ = envs_numpy(z1n, Zmix, zLo, i, j, L, b, r)
        key = ((pi >> (m - 1)) << m) | (pj >> (L - m))
        cs = []
        for k in np.unique(key):
            sel = key == k
            A = np.einsum("ea,ec->eac", h_new[m][sel], w_old[m][sel]).reshape(int(sel.sum()), r * r)
            cs.append(cond(A))
        out.append(np.array(cs))
    h_new, _ = envs_numpy(z1n, Zn, zLo, i, j, L, b, r)
    out.append(np.array([cond(h_new[L + 1][j == col]) for col in range(n) if np.any(j == col)]))
    return out
