"""Learned initializer: the MLP kernels against the float64 oracle, training,
and what the trained network gains over the low-rank start.

Tolerances: the kernels use BF16 weights (the oracle rounds the same way)
with FP32 activations and accumulation, so forward values and gradients are
compared at 1e-4 relative to the largest magnitude.
"""
import math

import numpy as np
import pytest

import paper_2510_17734_gb300 as bfc
import synth
import oracle
from oracle import gauge
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

DIMS = (2, 16, 40)


def identity_scaling(m, dims):
    bfc.bfc_mlp_set_scaling(m, -np.ones(dims[0]), np.ones(dims[0]), np.zeros(dims[2]), np.ones(dims[2]))


def test_forward_matches_oracle():
    with bfc.Mlp(*DIMS, seed=11) as m:
        identity_scaling(m.h, DIMS)
        x = np.random.default_rng(1).uniform(-1, 1, size=(5, 2))
        y = bfc.bfc_mlp_forward(m.h, x)
        p = bfc.bfc_mlp_get_params(m.h)
        yo = omlp.forward(p, DIMS, x, bf16=True)
        assert np.max(np.abs(y - yo)) <= 1e-4 * np.max(np.abs(yo))


@pytest.mark.parametrize("batch", [1, 7, 32])
def test_gradient_matches_oracle(batch):
    with bfc.Mlp(*DIMS, seed=12) as m:
        identity_scaling(m.h, DIMS)
        rng = np.random.default_rng(batch)
        x = rng.uniform(-1, 1, size=(batch, 2))
        t = rng.normal(size=(batch, DIMS[2]))
        g, loss = bfc.bfc_mlp_grad(m.h, x, t)
        p = bfc.bfc_mlp_get_params(m.h)
        lo, go = omlp.loss_and_grad(p, DIMS, x, t, bf16=True)
        assert abs(loss - lo) <= 1e-5 * lo
        assert np.max(np.abs(g - go)) <= 1e-4 * np.max(np.abs(go))


def test_large_output_layer_gradient_matches_oracle():
    dims = (2, 64, 5000)   # the tiled input-gradient reduction spans several CTAs
    with bfc.Mlp(*dims, seed=13) as m:
        identity_scaling(m.h, dims)
        rng = np.random.default_rng(4)
        x = rng.uniform(-1, 1, size=(9, 2))
        t = rng.normal(size=(9, dims[2]))
        g, loss = bfc.bfc_mlp_grad(m.h, x, t)
        lo, go = omlp.loss_and_grad(bfc.bfc_mlp_get_params(m.h), dims, x, t, bf16=True)
        assert abs(loss - lo) <= 1e-5 * lo
        assert np.max(np.abs(g - go)) <= 1e-4 * np.max(np.abs(go))


def test_training_fits_a_smooth_map():
    rng = np.random.default_rng(5)
    x = rng.uniform([0.1, 0.5], [0.3, 2.0], size=(64, 2))
    y = np.stack([np.sin(8 * x[:, 0]) * x[:, 1], np.cos(3 * x[:, 1]), x[:, 0] * x[:, 1]], axis=1)
    with bfc.Mlp(2, 64, 3, seed=3) as m:
        hist = bfc.bfc_mlp_train(m.h, x, y, epochs=300, batch=16, lr=3e-3, seed=9)
        assert hist[-1] < 0.02 * hist[0]
        pred = bfc.bfc_mlp_forward(m.h, x)
        assert np.sqrt(np.mean((pred - y) ** 2)) < 0.05 * np.sqrt(np.mean(y ** 2))


def test_invalid_model_arguments():
    with pytest.raises(bfc.BfcError, match="EINVAL"):
        bfc.bfc_mlp_create(0, 16, 4)
    with pytest.raises(bfc.BfcError, match="EINVAL"):
        bfc.bfc_mlp_create(2, 300, 4)
    with bfc.Mlp(2, 8, 4) as m:
        with pytest.raises(bfc.BfcError, match="EINVAL"):
            bfc.bfc_mlp_grad(m.h, np.zeros((33, 2)), np.zeros((33, 4)))
        with pytest.raises(bfc.BfcError, match="EINVAL"):
            bfc.bfc_mlp_train(m.h, np.zeros((4, 2)), np.zeros((4, 4)), epochs=1, batch=64)


# ------------------------------------------------------------- gauge fixing

@pytest.mark.parametrize("n,L,b,r", [(256, 4, 16, 4), (96, 4, 6, 5), (64, 0, 64, 3)])
def test_canonical_gauge_matches_oracle(n, L, b, r):
    rng = np.random.default_rng(n + r)
    P = oracle.num_params(n, L, b, r)
    X = rng.normal(size=P) + 1j * rng.normal(size=P)
    i, j = synth.draw_pairs(n, 500, 77)
    with bfc.Completion(n, L, b, r, 1e-6, i, j, np.ones(500, np.complex128), prec=bfc.PREC_FP64) as c:
        c.set_factors(X)
        c.canonicalize()
        C = c.get_factors()
        xg = c.eval(i, j)
    Co = gauge.canonicalize(n, L, b, r, X)
    assert np.max(np.abs(C - Co)) <= 1e-10 * np.max(np.abs(Co))
    xo = oracle.eval_entries(n, L, b, r, X, i, j)
    assert np.max(np.abs(xg - xo)) <= 1e-10 * np.max(np.abs(xo))


def test_canonicalize_needs_leaf_blocks_of_at_least_r_rows():
    i = np.zeros(4, np.int32)
    j = np.arange(4, dtype=np.int32)
    with bfc.Completion(16, 3, 2, 3, 1e-6, i, j, np.ones(4, np.complex128), prec=bfc.PREC_FP64) as c:
        with pytest.raises(bfc.BfcError, match="b >= r"):
            c.canonicalize()


# ---------------------------------------------------- learned start, small family

N, L, B, R = 256, 4, 16, 4


def family_problem(q, om, h):
    # n = 256 family: omega / (pi n) in [1/16, 1/6], h in [0.5, 2], |Omega| = 8 n log2 n;
    # every problem observes the same entry positions
    return synth.make_problem(f"fam{q}", N, L, B, R, om * math.pi * N, h, 8 * N * 8, 1e-8, 15, 0xBFC30000)


def make(p, **kw):
    return bfc.Completion(p.n, p.L, p.b, p.r, p.lam, p.i, p.j, p.t, p.it, p.jt, p.tt, prec=bfc.PREC_FP64, **kw)


def test_learned_start_beats_the_low_rank_start_on_held_out_problems():
    """Train on 96 gauge-fixed completions of the family, then start ALS on
    six held-out problems from the network and from the low-rank start."""
    rng = np.random.default_rng(21)
    X, Y = [], []
    for q in range(96):
        om, h = rng.uniform(1 / 16, 1 / 6), rng.uniform(0.5, 2.0)
        p = family_problem(q, om, h)
        with make(p, init_kind=1, seed=777, max_sweeps=15, tol=1e-12, lr_sweeps=10) as c:
            c.complete()
            c.canonicalize()
            Y.append(c.get_factors().view(np.float64).copy())
            X.append((om, h))
    X, Y = np.array(X), np.array(Y)
    with bfc.Mlp(2, 128, Y.shape[1], seed=5) as m:
        hist = bfc.bfc_mlp_train(m.h, X, Y, epochs=400, batch=16, lr=1e-3, seed=3)
        assert hist[-1] < 0.5 * hist[0]
        lr1, ml1, lr3, ml3 = [], [], [], []
        for q in range(6):
            om, h = rng.uniform(1 / 16, 1 / 6), rng.uniform(0.5, 2.0)
            p = family_problem(100 + q, om, h)
            with make(p, init_kind=1, seed=777, max_sweeps=3, tol=1e-12, lr_sweeps=10) as c:
                hist_lr = c.complete()
            with make(p) as c:
                used, err0 = bfc.bfc_init_learned(c.ctx, m.h, om * math.pi * N, h, allow_fallback=False)
                assert used and np.isfinite(err0)
                hist_ml = [c.sweep() for _ in range(3)]
            lr1.append(hist_lr[0]["train_rel_err"])
            ml1.append(hist_ml[0]["train_rel_err"])
            lr3.append(hist_lr[-1]["test_rel_err"])
            ml3.append(hist_ml[-1]["test_rel_err"])
        print("after 1 sweep (train):", np.round(ml1, 4), "low-rank", np.round(lr1, 4))
        print("after 3 sweeps (test):", np.round(ml3, 4), "low-rank", np.round(lr3, 4))
        assert np.median(ml1) < np.median(lr1)
        assert np.median(ml3) < np.median(lr3)
