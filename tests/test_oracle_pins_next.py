"""Pins of the oracle's first-order methods (Alg. 3/4 ADAM, Alg. 5 ADF with
the App. A.3 orthogonalization sweeps), of the randomized low-rank to
butterfly conversion (Alg. 2), of the dense matrix-vector product and of the
Radon workload, each against facts fixed by the paper or by mathematics,
independent of the code it checks:

* the right-to-left sweep keeps every entry, leaves the pinned orthonormality
  (zL leaf blocks Q^H Q = I, slice pairs [Z0 | Z1][Z0 | Z1]^H = I) and is
  unique (applying it twice changes nothing);
* with every entry observed the design of each ADF sub-step is orthonormal,
  so the exact line search lands on the block's regularized least-squares
  solution (checked against LAPACK for lambda = 0 and > 0), and with
  lambda = 0 one ADF iteration gives the same entries as one ALS sweep
  (Alg. 1) from the same state;
* ADAM: each factor's update equals the closed form of Alg. 3 applied to the
  gradient of the oracle's pinned gradient routine, taken at the newest
  point; with beta1 = beta2 = 0 and sigma = 0 it is sign descent;
* Alg. 2 reproduces an exact low-rank matrix A B^T (R <= r) to rounding;
* the matrix-vector product equals the whole-network einsum contraction
  applied to the vectors;
* the Radon matrix of Sec. 5.3 has the paper's closed form, and its
  complementary low-rank blocks have small numerical rank.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from helpers import split_packed
from oracle import first_order as fo
from oracle import lr2bf
from test_oracle_pins import dense_by_einsum


def _full(n):
    return synth.random_pairs_full(n)


# ------------------------------------------------------ orthogonalization

@pytest.mark.parametrize("n,L,b,r", [(64, 3, 8, 2), (96, 4, 6, 3), (40, 0, 40, 4), (64, 1, 32, 5)])
def test_right_to_left_sweep_keeps_entries_orthonormal_unique(n, L, b, r):
    X = synth.random_factors(n, L, r, 31 + n)
    i, j = _full(n)
    x0 = oracle.eval_entries(n, L, b, r, X, i, j)
    Y = fo.lr_orthogonalize(n, L, b, r, X)
    x1 = oracle.eval_entries(n, L, b, r, Y, i, j)
    assert np.abs(x1 - x0).max() <= 1e-12 * np.abs(x0).max()
    z1, Z, zL = split_packed(Y, n, L, b, r)
    if L == 0:
        np.testing.assert_allclose(zL.conj().T @ zL, np.eye(r), atol=1e-12)
    else:
        for p in range(n // b):
            blk = zL[p * b:(p + 1) * b]
            np.testing.assert_allclose(blk.conj().T @ blk, np.eye(r), atol=1e-12)
        for m in range(1, L + 1):
            for g in range(1 << L):
                M = np.hstack([Z[m - 1, 2 * g], Z[m - 1, 2 * g + 1]])
                np.testing.assert_allclose(M @ M.conj().T, np.eye(r), atol=1e-12)
    Y2 = fo.lr_orthogonalize(n, L, b, r, Y)
    assert np.abs(Y2 - Y).max() <= 1e-11 * np.abs(Y).max()


# --------------------------------------------------------------------- ADF

@pytest.mark.parametrize("n,L,b,r", [(64, 3, 8, 2), (48, 2, 12, 3), (32, 0, 32, 3)])
def test_adf_with_full_observation_equals_als_sweep(n, L, b, r):
    """lambda = 0: the least-squares fit of a block does not depend on the
    gauge, so one ADF iteration and one ALS sweep give the same entries."""
    X0 = synth.random_factors(n, L, r, 5 + n + L)
    i, j = _full(n)
    t = synth.helmholtz_line(n, 20.0, 1.0, i, j)
    Xa, res = fo.adf_iteration(n, L, b, r, 0.0, X0, i, j, t)
    Xs, _ = oracle.als_sweep(n, L, b, r, 0.0, X0, i, j, t)
    xa = oracle.eval_entries(n, L, b, r, Xa, i, j)
    xs = oracle.eval_entries(n, L, b, r, Xs, i, j)
    assert np.abs(xa - xs).max() <= 1e-10 * np.abs(xs).max()
    assert abs(res - np.linalg.norm(t - xa) / np.linalg.norm(t)) <= 1e-12


@pytest.mark.parametrize("lam", [0.0, 1e-3])
@pytest.mark.parametrize("n,L,b,r", [(64, 3, 8, 2), (32, 0, 32, 3)])
def test_adf_steps_are_block_least_squares_with_full_observation(n, L, b, r, lam):
    """Every ADF sub-step (with lambda > 0 too) lands on the exact regularized
    least-squares solution of its blocks, computed here by LAPACK from the
    design of the state before the step: with every entry observed the
    design is orthonormal, where one exact line search along the gradient is
    the solve."""
    from helpers import envs_numpy, lstsq_block
    X0 = synth.random_factors(n, L, r, 15 + n + L)
    i, j = _full(n)
    t = synth.helmholtz_line(n, 20.0, 1.0, i, j)
    trace = []
    fo.adf_iteration(n, L, b, r, lam, X0, i, j, t, trace=trace)
    assert [lv for lv, _, _ in trace] == list(range(L + 2))
    pi, pj = i // b, j // b
    for lev, before, after in trace:
        z1b, Zb, zLb = split_packed(before, n, L, b, r)
        z1a, Za, zLa = split_packed(after, n, L, b, r)
        h, w = envs_numpy(z1b, Zb, zLb, i, j, L, b, r)
        if lev == 0:
            for row in range(0, n, 7):
                sel = np.nonzero(i == row)[0]
                want = lstsq_block(w[0][sel], t[sel], lam)
                np.testing.assert_allclose(z1a[row], want, rtol=0, atol=1e-10 * np.abs(want).max())
        elif lev == L + 1:
            for col in range(0, n, 7):
                sel = np.nonzero(j == col)[0]
                want = lstsq_block(h[L + 1][sel], t[sel], lam)
                np.testing.assert_allclose(zLa[col], want, rtol=0, atol=1e-10 * np.abs(want).max())
        else:
            key = ((pi >> (lev - 1)) << lev) | (pj >> (L - lev))
            for k in range(0, 1 << (L + 1), 5):
                sel = np.nonzero(key == k)[0]
                A = np.einsum("ea,ec->eac", h[lev][sel], w[lev][sel]).reshape(len(sel), r * r)
                want = lstsq_block(A, t[sel], lam)
                np.testing.assert_allclose(Za[lev - 1, k].ravel(), want, rtol=0,
                                           atol=1e-10 * np.abs(want).max())


def test_adf_objective_decreases_on_partial_observation():
    p = synth.config(1)
    A, B = synth.random_lowrank_start(p, p.r)
    A, B = oracle.lr_complete(p.n, p.r, p.lam, A, B, p.i, p.j, p.t, 10)
    X = oracle.embed_lowrank(p.n, p.L, p.b, p.r, A, B)
    f = oracle.objective(p.n, p.L, p.b, p.r, p.lam, X, p.i, p.j, p.t)
    for _ in range(6):
        X, res = fo.adf_iteration(p.n, p.L, p.b, p.r, p.lam, X, p.i, p.j, p.t)
        f1 = oracle.objective(p.n, p.L, p.b, p.r, p.lam, X, p.i, p.j, p.t)
        assert f1 <= f * (1 + 1e-12)
        assert abs(res - oracle.rel_err(p.n, p.L, p.b, p.r, X, p.i, p.j, p.t)) <= 1e-10
        f = f1


# -------------------------------------------------------------------- ADAM

def _factor_slices(n, L, r):
    """Packed index ranges of the factors S^1, S^2 .. S^{L+1}, S^{L+2}."""
    S = 1 << (L + 1)
    out = [slice(0, n * r)]
    off = n * r
    for _ in range(L):
        out.append(slice(off, off + S * r * r))
        off += S * r * r
    out.append(slice(off, off + n * r))
    return out


@pytest.mark.parametrize("n,L,b,r", [(32, 2, 8, 2), (24, 0, 24, 3)])
def test_adam_iteration_is_alg3_on_pinned_gradients(n, L, b, r):
    lam = 1e-2
    X0 = synth.random_factors(n, L, r, 9 + n)
    i, j = synth.draw_pairs(n, 300, 4 + n)
    t = synth.helmholtz_line(n, 15.0, 1.0, i, j)
    P = X0.size
    alpha, b1, b2, sig = 2e-2, 0.8, 0.95, 1e-8
    M = synth.SplitMix64(3).normal(2 * P).reshape(P, 2) * 0.1
    V = np.abs(synth.SplitMix64(4).normal(2 * P).reshape(P, 2)) * 0.1
    it = 3
    got = fo.adam_iteration(n, L, b, r, lam, X0, i, j, t, M.copy(), V.copy(), it, alpha, b1, b2, sig)
    want = X0.copy()
    Mw, Vw = M.copy(), V.copy()
    for sl in _factor_slices(n, L, r):
        g, _ = oracle.grad(n, L, b, r, lam, want, i, j, t, include_reg=True)
        gr = np.stack([g[sl].real, g[sl].imag], axis=-1)
        Mw[sl] = b1 * Mw[sl] + (1 - b1) * gr
        Vw[sl] = b2 * Vw[sl] + (1 - b2) * gr ** 2
        step = alpha * (Mw[sl] / (1 - b1 ** it)) / (np.sqrt(Vw[sl] / (1 - b2 ** it)) + sig)
        want[sl] = want[sl] - (step[:, 0] + 1j * step[:, 1])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_adam_without_moments_is_sign_descent():
    n, L, b, r = 32, 2, 8, 2
    X0 = synth.random_factors(n, L, r, 77)
    i, j = synth.draw_pairs(n, 200, 78)
    t = synth.helmholtz_line(n, 9.0, 1.0, i, j)
    P = X0.size
    got = fo.adam_iteration(n, L, b, r, 0.0, X0, i, j, t, np.zeros((P, 2)), np.zeros((P, 2)), 1,
                            alpha=0.01, beta1=0.0, beta2=0.0, sigma=0.0)
    # S^1 is updated first, at the start point: its step is -alpha sign(grad)
    g, _ = oracle.grad(n, L, b, r, 0.0, X0, i, j, t, include_reg=False)
    sl = slice(0, n * r)
    want = X0[sl] - 0.01 * (np.sign(g[sl].real) + 1j * np.sign(g[sl].imag))
    np.testing.assert_allclose(got[sl], want, rtol=0, atol=1e-15)


# ------------------------------------------------------------------ Alg. 2

@pytest.mark.parametrize("n,L,b,r,R,p", [(64, 2, 16, 4, 4, 5), (128, 3, 16, 4, 3, 5), (256, 4, 16, 6, 6, 3),
                                         (32, 0, 32, 3, 3, 2), (64, 1, 32, 4, 4, 5), (512, 5, 16, 8, 8, 5),
                                         (64, 4, 4, 12, 10, 5), (128, 5, 4, 12, 12, 5)])
def test_alg2_reproduces_exact_low_rank(n, L, b, r, R, p):
    rng = synth.SplitMix64(7 + n + R)
    A = rng.cnormal(n * R).reshape(n, R)
    B = rng.cnormal(n * R).reshape(n, R)
    G = synth.lr2bf_gaussians(n, L, b, r, p, 99 + n)
    X = lr2bf.lr_to_butterfly(n, L, b, r, A, B, G, p)
    assert X.size == oracle.num_params(n, L, b, r)
    i, j = _full(n)
    x = oracle.eval_entries(n, L, b, r, X, i, j).reshape(n, n)
    T = A @ B.T
    assert np.abs(x - T).max() <= 1e-12 * np.abs(T).max()
    # the outer factors are orthonormal bases of the leaf blocks (z1 only
    # when the middle level is not z1 itself)
    # b >= r: the leaf blocks of z1 and zL are orthonormal bases (z1 only when
    # the middle level is not z1 itself); b < r: their b columns are, and the
    # rest are zero
    z1, _, zL = split_packed(X, n, L, b, r)
    k = min(b, r)
    eye = np.zeros((r, r))
    eye[:k, :k] = np.eye(k)
    for q in range(n // b):
        blk = zL[q * b:(q + 1) * b]
        np.testing.assert_allclose(blk.conj().T @ blk, eye, atol=1e-12)
        if L >= 2:
            blk = z1[q * b:(q + 1) * b]
            np.testing.assert_allclose(blk.conj().T @ blk, eye, atol=1e-12)


def test_alg2_gaussian_layout_matches_synth():
    n, L, b, r, p = 256, 4, 16, 6, 3
    rows, cols = lr2bf.gaussian_layout(n, L, b, r, p)
    assert synth.lr2bf_gaussians(n, L, b, r, p, 1).size == sum(rows) * cols
    assert rows == [256, 128, 64, 128, 64]


# ------------------------------------------------------------------ matvec

@pytest.mark.parametrize("L,b,r,nvec", [(0, 6, 2, 1), (2, 3, 2, 3), (3, 2, 3, 2), (4, 2, 2, 1)])
def test_matvec_equals_einsum_network_times_vectors(L, b, r, nvec):
    n = b << L
    X = synth.random_factors(n, L, r, 13 + L)
    V = synth.SplitMix64(14 + L).cnormal(n * nvec).reshape(n, nvec)
    U = oracle.matvec(n, L, b, r, X, V)
    D = dense_by_einsum(X, n, L, b, r)
    np.testing.assert_allclose(U, D @ V, rtol=0, atol=1e-12 * np.abs(D @ V).max())


# ------------------------------------------------------------------- Radon

def test_radon_closed_form_and_butterfly_structure():
    n = 256
    i, j = _full(n)
    T = synth.radon_1d(n, i, j).reshape(n, n)
    # closed form at a few points (1-based x = i'/n, y = j' - n/2)
    for (a, c) in [(0, 0), (5, 200), (255, 127), (128, 128)]:
        x, y = (a + 1) / n, (c + 1) - n / 2
        phi = x * y + (2 + math.sin(2 * math.pi * x)) / 8 * abs(y)
        assert abs(T[a, c] - np.exp(2j * math.pi * phi)) <= 1e-12
    assert np.allclose(np.abs(T), 1.0)
    # complementary low-rank: blocks of a level-l partition have small
    # numerical rank (well below the block size), the whole matrix does not
    L, b = 6, 4
    for lev in (2, 3, 4):
        rows, cols = n >> lev, n >> (L - lev)
        ranks = []
        for bi in range(1 << lev):
            for bj in range(0, 1 << (L - lev), 7):
                sv = np.linalg.svd(T[bi * rows:(bi + 1) * rows, bj * cols:(bj + 1) * cols], compute_uv=False)
                ranks.append(int(np.sum(sv > 1e-3 * sv[0])))
        assert max(ranks) <= 16 < min(rows, cols) * 2
    sv = np.linalg.svd(T, compute_uv=False)
    assert np.sum(sv > 1e-3 * sv[0]) > n // 2
