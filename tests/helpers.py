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
