"""Parity of the randomized low-rank to butterfly conversion (Alg. 2) on the
GPU (bfc_lowrank_to_butterfly, and bfc_complete's init_kind 2) with the
oracle's Alg. 2 (oracle.lr2bf), on the same caller-drawn Gaussians.

FP64 throughout: entries of the butterfly against A B^T and against the
oracle's butterfly at 1e-10 relative (measured against max(|x_ref|,
rms(x_ref))); with R = r the sketches of every block have full rank, the
column pivots and hence the factors themselves are the same on both sides.
"""
import numpy as np
import pytest

import oracle
import paper_2510_17734_gb300 as bfc
import synth
from helpers import rel_dev
from oracle import lr2bf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,L,b,r,R,p", [(256, 4, 16, 4, 4, 5), (1024, 6, 16, 6, 3, 5), (512, 5, 16, 8, 8, 5),
                                         (64, 0, 64, 4, 4, 3), (128, 1, 64, 5, 5, 2), (4096, 8, 16, 6, 6, 5),
                                         (1024, 8, 4, 12, 10, 5), (256, 6, 4, 12, 12, 3)])
def test_lr2bf_parity(n, L, b, r, R, p):
    rng = synth.SplitMix64(101 + n + R)
    A = rng.cnormal(n * R).reshape(n, R)
    B = rng.cnormal(n * R).reshape(n, R)
    G = synth.lr2bf_gaussians(n, L, b, r, p, 202 + n)
    Xo = lr2bf.lr_to_butterfly(n, L, b, r, A, B, G, p)
    i, j = synth.draw_pairs(n, min(n * n, 20 * n), 7)
    t = (A[i] * B[j]).sum(axis=1)
    with bfc.Completion(n, L, b, r, 1e-8, i, j, t) as c:
        c.lowrank_to_butterfly(A, B, p, G)
        Xg = c.get_factors()
        xg = c.eval(i, j)
    assert rel_dev(xg, t) <= 1e-10                      # reproduces A B^T
    xo = oracle.eval_entries(n, L, b, r, Xo, i, j)
    assert rel_dev(xg, xo) <= 1e-10
    if R == r and b >= r:
        # full-rank pivots everywhere: the factors are unique (a rank-deficient
        # step completes Q with arbitrary orthonormal columns, chosen
        # differently by LAPACK and by the warp QR)
        assert rel_dev(Xg, Xo) <= 1e-8


def test_lr2bf_rejects_bad_arguments():
    n, L, b, r = 64, 2, 16, 4
    i, j = synth.draw_pairs(n, 300, 3)
    t = synth.helmholtz_line(n, 5.0, 1.0, i, j)
    A = np.ones((n, 2), np.complex128)
    G = synth.lr2bf_gaussians(n, L, b, r, 40, 1)
    with bfc.Completion(n, L, b, r, 1e-8, i, j, t) as c:
        with pytest.raises(bfc.BfcError, match="EINVAL"):
            c.lowrank_to_butterfly(A, A, 40, G)             # r + p > 32
        with pytest.raises(bfc.BfcError, match="EINVAL"):
            c.lowrank_to_butterfly(np.ones((n, 5), np.complex128), np.ones((n, 5), np.complex128), 2, G)


@pytest.mark.parametrize("prec", [bfc.PREC_FP64, bfc.PREC_C64])
def test_complete_init_kind_2_is_lowrank_completion_then_alg2(prec):
    """bfc_complete's start with init_kind 2: low-rank completion (Alg. 1
    with L = 0, R = r, 10 sweeps from the SplitMix64 start of params.seed)
    converted by Alg. 2 with the Gaussians of SplitMix64(seed + 1).  The
    oracle runs the same two steps; the entries of the starts agree."""
    p = synth.config(1)
    seed = p.seed + synth.SEED_INIT
    A0, B0 = synth.random_lowrank_start(p, p.r)
    A, B = oracle.lr_complete(p.n, p.r, p.lam, A0, B0, p.i, p.j, p.t, 10)
    G = synth.lr2bf_gaussians(p.n, p.L, p.b, p.r, 5, seed + 1)
    Xo = lr2bf.lr_to_butterfly(p.n, p.L, p.b, p.r, A, B, G, 5)
    with bfc.Completion(p.n, p.L, p.b, p.r, p.lam, p.i, p.j, p.t, p.it, p.jt, p.tt, prec=prec, max_sweeps=0,
                        seed=seed, init_kind=2, lr_sweeps=10) as c:
        c.complete()
        Xg = c.get_factors()
        hist = c.complete()   # further sweeps from the converted start work as usual
    for (ii, jj) in [(p.i, p.j), (p.it, p.jt)]:
        xg = oracle.eval_entries(p.n, p.L, p.b, p.r, Xg, ii, jj)
        xo = oracle.eval_entries(p.n, p.L, p.b, p.r, Xo, ii, jj)
        assert rel_dev(xg, xo) <= (1e-8 if prec == bfc.PREC_FP64 else 1e-4)
    assert hist == [] or hist[-1]["train_rel_err"] < 1.0
