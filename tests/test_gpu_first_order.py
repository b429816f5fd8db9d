"""Parity of the first-order methods and of the butterfly matrix-vector
product (CUDA path through the C ABI) with the oracle.

* bfc_matvec (Eq. butterfly-mat-vec) against the oracle's u_i = sum_j x_ij v_j
  (complex128 definition), and at n = 65536 column by column against the
  oracle's entry evaluation (X e_j is column j of X);
* bfc_adam (Alg. 3/4) against oracle.first_order.adam_iteration;
* bfc_adf (Alg. 5, App. A.3) against oracle.first_order.adf_iteration: after
  every iteration all factors but S^{L+2} are left-orthonormal (the gauge is
  fixed), so factors are compared as well as entries.

Tolerances: FP64 path 1e-10 relative on entry values (measured against
max(|x_ref|, rms(x_ref))); complex64 path 1e-4.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2510_17734_gb300 as bfc
import synth
from helpers import rel_dev
from oracle import first_order as fo

pytestmark = pytest.mark.gpu

TOL = {bfc.PREC_FP64: 1e-10, bfc.PREC_C64: 1e-4}
PRECS = [bfc.PREC_FP64, bfc.PREC_C64]


def lr_start(p, sweeps=10):
    A, B = synth.random_lowrank_start(p, p.r)
    A, B = oracle.lr_complete(p.n, p.r, p.lam, A, B, p.i, p.j, p.t, sweeps)
    return oracle.embed_lowrank(p.n, p.L, p.b, p.r, A, B)


def make(p, prec, **kw):
    return bfc.Completion(p.n, p.L, p.b, p.r, p.lam, p.i, p.j, p.t, p.it, p.jt, p.tt, prec=prec, **kw)


@pytest.fixture(scope="module")
def cfg1():
    p = synth.config(1)
    return p, lr_start(p)


@pytest.fixture(scope="module")
def cfg2s():
    p = synth.config(2, n_override=1024)
    return p, lr_start(p)


# ------------------------------------------------------------------ matvec

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", [(256, 4, 16, 4), (1024, 6, 16, 6), (48, 0, 48, 3), (96, 4, 6, 5),
                                   (24, 3, 3, 2), (128, 3, 16, 7)])
@pytest.mark.parametrize("nvec", [1, 5])
def test_matvec_parity(prec, shape, nvec):
    n, L, b, r = shape
    X = synth.random_factors(n, L, r, 21 + n + L)
    V = synth.SplitMix64(22 + n).cnormal(n * nvec).reshape(n, nvec)
    i, j = synth.draw_pairs(n, min(n * n, 4 * n), 23)
    t = synth.helmholtz_line(n, 5.0, 1.0, i, j)
    with bfc.Completion(n, L, b, r, 1e-8, i, j, t, prec=prec) as c:
        c.set_factors(X)
        U = c.matvec(V)
    with oracle.threads(oracle.max_threads()):
        Uo = oracle.matvec(n, L, b, r, X, V)
    assert rel_dev(U, Uo) <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_matvec_full_size_columns(prec):
    """n = 65536 (L = 12, r = 8): X e_j is column j of X; two columns per
    call, checked against the oracle's evaluation of every entry of them."""
    p = synth.config(3)
    X = synth.random_factors(p.n, p.L, p.r, 31, sigma=0.5)
    cols = [5, 40000]
    V = np.zeros((p.n, len(cols)), dtype=np.complex128)
    for q, jc in enumerate(cols):
        V[jc, q] = 1.0
    with make(p, prec) as c:
        c.set_factors(X)
        U = c.matvec(V)
    rows = np.arange(p.n, dtype=np.int32)
    with oracle.threads(oracle.max_threads()):
        for q, jc in enumerate(cols):
            want = oracle.eval_entries(p.n, p.L, p.b, p.r, X, rows, np.full(p.n, jc, np.int32))
            assert rel_dev(U[:, q], want) <= TOL[prec]


def test_matvec_rejects_bad_nvec(cfg1):
    p, X = cfg1
    with make(p, bfc.PREC_FP64) as c:
        with pytest.raises(bfc.BfcError, match="EINVAL"):
            bfc.bfc_matvec(c.ctx, 0, np.zeros(2, np.complex128), np.zeros(2, np.complex128))


# -------------------------------------------------------------------- ADAM

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("which", ["cfg1", "cfg2s"])
def test_adam_parity(request, which, prec):
    p, X0 = request.getfixturevalue(which)
    iters, alpha = 3, 2e-3
    P = X0.size
    M, V = np.zeros((P, 2)), np.zeros((P, 2))
    Xo = X0
    objs = []
    for it in range(1, iters + 1):
        Xo = fo.adam_iteration(p.n, p.L, p.b, p.r, p.lam, Xo, p.i, p.j, p.t, M, V, it, alpha=alpha)
        objs.append(oracle.objective(p.n, p.L, p.b, p.r, p.lam, Xo, p.i, p.j, p.t))
    with make(p, prec, tol=0.0) as c:
        c.set_factors(X0)
        hist = c.adam(iters, alpha=alpha)
        Xg = c.get_factors()
    assert len(hist) == iters
    for h, fo_ in zip(hist, objs):
        assert abs(h["objective"] - fo_) <= TOL[prec] * abs(fo_)
    for (ii, jj) in [(p.i, p.j), (p.it, p.jt)]:
        xg = oracle.eval_entries(p.n, p.L, p.b, p.r, Xg, ii, jj)
        xo = oracle.eval_entries(p.n, p.L, p.b, p.r, Xo, ii, jj)
        assert rel_dev(xg, xo) <= TOL[prec]


def test_adam_decreases_objective(cfg1):
    p, X0 = cfg1
    with make(p, bfc.PREC_FP64, tol=0.0) as c:
        c.set_factors(X0)
        f0 = oracle.objective(p.n, p.L, p.b, p.r, p.lam, X0, p.i, p.j, p.t)
        hist = c.adam(20, alpha=1e-3)
    assert hist[-1]["objective"] < f0
    assert hist[-1]["objective"] < hist[0]["objective"]


# --------------------------------------------------------------------- ADF

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("which", ["cfg1", "cfg2s"])
def test_adf_parity(request, which, prec):
    p, X0 = request.getfixturevalue(which)
    iters = 3
    Xo, res = X0, []
    for _ in range(iters):
        Xo, e = fo.adf_iteration(p.n, p.L, p.b, p.r, p.lam, Xo, p.i, p.j, p.t)
        res.append(e)
    with make(p, prec, tol=0.0) as c:
        c.set_factors(X0)
        hist = c.adf(iters)
        Xg = c.get_factors()
    assert len(hist) == iters
    for h, e in zip(hist, res):
        assert abs(h["train_rel_err"] - e) <= TOL[prec] * e
    for (ii, jj) in [(p.i, p.j), (p.it, p.jt)]:
        xg = oracle.eval_entries(p.n, p.L, p.b, p.r, Xg, ii, jj)
        xo = oracle.eval_entries(p.n, p.L, p.b, p.r, Xo, ii, jj)
        assert rel_dev(xg, xo) <= TOL[prec]
    if prec == bfc.PREC_FP64:
        # the QR sweeps fix the gauge: the factors themselves agree
        assert rel_dev(Xg, Xo) <= 1e-8


@pytest.mark.parametrize("n,L,b,r", [(48, 0, 48, 3), (64, 3, 8, 2), (96, 2, 24, 5), (128, 1, 64, 8)])
def test_adf_odd_shapes(n, L, b, r):
    X0 = synth.random_factors(n, L, r, 41 + n)
    i, j = synth.draw_pairs(n, min(n * n, 8 * n * max(1, L) + 11), 42 + n)
    t = synth.helmholtz_line(n, math.pi * n / 8, 1.0, i, j)
    lam = 1e-6
    Xo = X0
    for _ in range(2):
        Xo, _ = fo.adf_iteration(n, L, b, r, lam, Xo, i, j, t)
    with bfc.Completion(n, L, b, r, lam, i, j, t, prec=bfc.PREC_FP64, tol=0.0) as c:
        c.set_factors(X0)
        c.adf(2)
        Xg = c.get_factors()
    xg = oracle.eval_entries(n, L, b, r, Xg, i, j)
    xo = oracle.eval_entries(n, L, b, r, Xo, i, j)
    assert rel_dev(xg, xo) <= 1e-10


def test_adf_monotone_and_rejects_small_leaves(cfg1):
    p, X0 = cfg1
    with make(p, bfc.PREC_FP64, tol=0.0) as c:
        c.set_factors(X0)
        hist = c.adf(8)
    objs = [h["objective"] for h in hist]
    assert all(b_ <= a_ * (1 + 1e-10) for a_, b_ in zip(objs[:-1], objs[1:]))
    i, j = synth.draw_pairs(64, 400, 3)
    t = synth.helmholtz_line(64, 5.0, 1.0, i, j)
    with bfc.Completion(64, 4, 4, 6, 1e-6, i, j, t) as c:     # b = 4 < r = 6
        with pytest.raises(bfc.BfcError, match="b >= r"):
            c.adf(1)
