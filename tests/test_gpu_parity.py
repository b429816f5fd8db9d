"""Parity of the CUDA path (through the C ABI) with the complex128 oracle.

Tolerances (from the precision of each path): integer work (decoding, entry
orderings) bit-exact; FP64 path 1e-10 relative on entry values and the
objective; complex64 precision form 1e-4 relative.  The precision form
solves every system with the ridge floor lambda_eff = max(lambda,
2^-20 trace(K) / dim) (its reading of the regularization); it is compared
with the oracle run under the same reading (oracle.als_sweep(ridge_rel=2^-20)),
and its distance to the plain oracle is checked to be that of the reading
itself plus the tolerance.  On deliberately ill-conditioned small problems
(few observations per block) the complex64 tolerance is
max(1e-4, kappa_max 2^-24): complex64 rounding amplified by the largest
condition number of the sweep's block systems (measured ratio of deviation
to that bound <= 0.2).  Relative deviations of
entry values are measured against max(|x_ref|, rms(x_ref)) so that entries
near zero do not dominate.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2510_17734_gb300 as bfc
import synth
from helpers import (block_conditions, block_objective, envs_numpy, level_keys, lstsq_block, rel_dev,
                     split_packed)

pytestmark = pytest.mark.gpu

TOL = {bfc.PREC_FP64: 1e-10, bfc.PREC_C64: 1e-4}
PRECS = [bfc.PREC_FP64, bfc.PREC_C64]
RIDGE = {bfc.PREC_FP64: 0.0, bfc.PREC_C64: 2.0 ** -20}   # the ridge floor each path solves with


def oracle_sweep(p, X0, prec, lam=None, t=None):
    """The oracle's sweep under the regularization reading of `prec`."""
    lam = p.lam if lam is None else lam
    t = p.t if t is None else t
    return oracle.als_sweep(p.n, p.L, p.b, p.r, lam, X0, p.i, p.j, t, ridge_rel=RIDGE[prec])


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
    # the n = 4096 workload's structure (b = 16, r = 6, 6 n log2 n samples,
    # noise) at n = 1024 so the oracle finishes in seconds
    p = synth.config(2, n_override=1024)
    return p, lr_start(p)


# ------------------------------------------------------------- integers

def test_decode_bit_exact_exhaustive_small():
    for (n, L, b) in [(64, 4, 4), (48, 4, 3), (32, 0, 32), (16, 4, 1)]:
        i, j = synth.random_pairs_full(n)
        keys = bfc.bfc_decode(n, L, b, i, j)
        for e in range(0, len(i), 7):
            want = [int(i[e])] + [oracle.slice_id(i[e], j[e], m, L, b) for m in range(1, L + 1)] + [int(j[e])]
            assert list(keys[e]) == want


def test_decode_bit_exact_large_sample():
    n, L, b = 65536, 12, 16
    i, j = synth.draw_pairs(n, 3000, 17)
    keys = bfc.bfc_decode(n, L, b, i, j)
    for e in range(len(i)):
        want = [int(i[e])] + [oracle.slice_id(i[e], j[e], m, L, b) for m in range(1, L + 1)] + [int(j[e])]
        assert list(keys[e]) == want


@pytest.mark.parametrize("group_ratio", [0.0, 2.0, -1.0])
def test_orders_are_stable_sorts(cfg1, group_ratio):
    """Level orders: stable sorts of the entries by row, by the oracle's slice
    id of S^{m+1} and by column; inside a slice of a middle level that runs
    the grouped Gram the entries are further ordered by their row (levels
    with 2m <= L + 1) or column (the groups that share an environment),
    stably; the other middle levels keep input order inside a slice."""
    p, X0 = cfg1
    with make(p, bfc.PREC_C64, group_ratio=group_ratio) as c:
        n_grouped = 0
        for level in range(p.L + 2):
            sub = np.zeros(p.nnz, dtype=np.int64)
            if level == 0:
                key = p.i.astype(np.int64)
            elif level == p.L + 1:
                key = p.j.astype(np.int64)
            else:
                key = np.array([oracle.slice_id(a, b_, level, p.L, p.b) for a, b_ in zip(p.i, p.j)])
                other = (p.j if 2 * level > p.L + 1 else p.i).astype(np.int64)
                ngroups, grouped = c.level_groups(level)
                # groups: distinct (slice, row) or (slice, column) pairs
                assert ngroups == np.unique(key * p.n + other).size
                if grouped:
                    sub = other
                    n_grouped += 1
            perm, seg = c.order(level)
            np.testing.assert_array_equal(perm, np.lexsort((sub, key)))   # stable, key then sub
            K = p.n if level in (0, p.L + 1) else 1 << (p.L + 1)
            np.testing.assert_array_equal(seg, np.searchsorted(np.sort(key), np.arange(K + 1)))
        if group_ratio == 2.0:
            assert n_grouped == p.L
        elif group_ratio < 0:
            assert n_grouped == 0


# ------------------------------------------------------------------ eval

@pytest.mark.parametrize("prec", PRECS)
def test_eval_parity(cfg2s, prec):
    p, _ = cfg2s
    X = synth.random_factors(p.n, p.L, p.r, 5)
    with make(p, prec) as c:
        c.set_factors(X)
        np.testing.assert_array_equal(c.get_factors(), X)
        got = c.eval(p.i, p.j)
    want = oracle.eval_entries(p.n, p.L, p.b, p.r, X, p.i, p.j)
    assert rel_dev(got, want) <= TOL[prec]


# ------------------------------------------------------------- ALS sweep

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("which", ["cfg1", "cfg2s"])
def test_one_sweep_parity(request, which, prec):
    p, X0 = request.getfixturevalue(which)
    Xo, st_o = oracle_sweep(p, X0, prec)
    with make(p, prec) as c:
        c.set_factors(X0)
        c.profile(True)
        st = c.sweep()
        prof = c.profile_read()
        Xg = c.get_factors()
    tol = TOL[prec]
    assert abs(st["objective"] - st_o["objective"]) <= tol * abs(st_o["objective"])
    assert abs(st["train_rel_err"] - st_o["train_rel_err"]) <= tol * st_o["train_rel_err"]
    te_o = oracle.rel_err(p.n, p.L, p.b, p.r, Xo, p.it, p.jt, p.tt)
    assert abs(st["test_rel_err"] - te_o) <= tol * te_o
    assert st["singular_slices"] == st_o["singular"] == 0
    # entries of the two results agree on both the training and test sets
    for (ii, jj) in [(p.i, p.j), (p.it, p.jt)]:
        xg = oracle.eval_entries(p.n, p.L, p.b, p.r, Xg, ii, jj)
        xo = oracle.eval_entries(p.n, p.L, p.b, p.r, Xo, ii, jj)
        assert rel_dev(xg, xo) <= tol
    if prec == bfc.PREC_FP64:
        # with lambda > 0 every block is strictly convex: the factors are unique
        assert rel_dev(Xg, Xo) <= 1e-9
    else:
        # distance to the plain-lambda oracle = the ridge reading's own effect
        Xp, _ = oracle.als_sweep(p.n, p.L, p.b, p.r, p.lam, X0, p.i, p.j, p.t)
        xg = oracle.eval_entries(p.n, p.L, p.b, p.r, Xg, p.it, p.jt)
        xp = oracle.eval_entries(p.n, p.L, p.b, p.r, Xp, p.it, p.jt)
        xo = oracle.eval_entries(p.n, p.L, p.b, p.r, Xo, p.it, p.jt)
        assert rel_dev(xg, xp) <= rel_dev(xo, xp) + tol
    # kernels per sweep: 1 + L right environments, 3 + 3 outer fiber kernels,
    # per middle level Gram + solve (+ the FP64 fallback, which also counts
    # the level's fallbacks, in the precision form), residual reduction, 2 for
    # ||S||^2, 2 for the test error;
    # a middle level on the grouped Gram runs two kernels for its Gram
    per_level = 3 if prec == bfc.PREC_C64 else 2
    n_grouped = prof.get("mid_gram_grp", (0, 0.0))[0] // 2
    assert st["launches"] == 12 + (1 + per_level) * p.L + n_grouped


@pytest.fixture(scope="module")
def cfg3s():
    # the n = 65536 workload's structure (b = 16, r = 8, 4 n log2 n samples)
    # at n = 2048: the rank-8 middle levels run the 64-feature Gram
    p = synth.config(3, n_override=2048)
    return p, lr_start(p)


@pytest.mark.parametrize("gram", [bfc.GRAM_AUTO, bfc.GRAM_TENSOR, bfc.GRAM_CUDA])
def test_one_sweep_parity_rank8_gram_kernels(cfg3s, gram):
    """The middle-level Gram kernels of the precision form (grouped by row /
    column at the outer levels with tensor cores elsewhere; tensor cores per
    entry: three-term TF32 products; CUDA cores per entry: complex64 FMA)
    against the oracle sweep, with the complex64 tolerance."""
    p, X0 = cfg3s
    Xo, st_o = oracle_sweep(p, X0, bfc.PREC_C64)
    with make(p, bfc.PREC_C64, gram_impl=gram) as c:
        c.set_factors(X0)
        st = c.sweep()
        Xg = c.get_factors()
    tol = TOL[bfc.PREC_C64]
    assert abs(st["objective"] - st_o["objective"]) <= tol * abs(st_o["objective"])
    assert abs(st["train_rel_err"] - st_o["train_rel_err"]) <= tol * st_o["train_rel_err"]
    for (ii, jj) in [(p.i, p.j), (p.it, p.jt)]:
        xg = oracle.eval_entries(p.n, p.L, p.b, p.r, Xg, ii, jj)
        xo = oracle.eval_entries(p.n, p.L, p.b, p.r, Xo, ii, jj)
        assert rel_dev(xg, xo) <= tol


def test_gram_kernels_agree_over_sweeps(cfg3s):
    """Five sweeps with each Gram kernel follow the same trajectory."""
    p, X0 = cfg3s
    hist = {}
    for gram in (bfc.GRAM_AUTO, bfc.GRAM_TENSOR, bfc.GRAM_CUDA):
        with make(p, bfc.PREC_C64, gram_impl=gram) as c:
            c.set_factors(X0)
            hist[gram] = [c.sweep()["train_rel_err"] for _ in range(5)]
    for g in (bfc.GRAM_AUTO, bfc.GRAM_TENSOR):
        for a, b in zip(hist[g], hist[bfc.GRAM_CUDA]):
            assert abs(a - b) <= 1e-4 * b


@pytest.mark.parametrize("gram", [bfc.GRAM_AUTO, bfc.GRAM_TENSOR, bfc.GRAM_CUDA])
@pytest.mark.parametrize("scale", [1e-6, 1e6])
def test_rank8_gram_far_from_unit_scale(cfg3s, scale, gram):
    """Data far from unit size keeps the complex64 parity of both Gram
    kernels.  The problem is the unit-size one scaled exactly: values and
    starting outer factors times `scale`, lambda times scale^2 (the
    environments, the features and the right-hand sides scale with the data,
    the middle slices do not)."""
    p, X0 = cfg3s
    X1 = X0.copy()
    X1[:p.n * p.r] *= scale   # z1 leads the packed factors
    t, tt, lam = p.t * scale, p.tt * scale, p.lam * scale * scale
    Xo, st_o = oracle.als_sweep(p.n, p.L, p.b, p.r, lam, X1, p.i, p.j, t, ridge_rel=RIDGE[bfc.PREC_C64])
    with bfc.Completion(p.n, p.L, p.b, p.r, lam, p.i, p.j, t, p.it, p.jt, tt,
                        prec=bfc.PREC_C64, gram_impl=gram) as c:
        c.set_factors(X1)
        st = c.sweep()
        Xg = c.get_factors()
    tol = TOL[bfc.PREC_C64]
    assert abs(st["objective"] - st_o["objective"]) <= tol * abs(st_o["objective"])
    assert abs(st["train_rel_err"] - st_o["train_rel_err"]) <= tol * st_o["train_rel_err"]
    xg = oracle.eval_entries(p.n, p.L, p.b, p.r, Xg, p.it, p.jt)
    xo = oracle.eval_entries(p.n, p.L, p.b, p.r, Xo, p.it, p.jt)
    assert rel_dev(xg, xo) <= tol


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("which", ["cfg1", "cfg3s"])
def test_grouped_gram_equals_per_entry_gram(request, which, prec):
    """The grouped Gram (entries of one row / column of a slice share an
    environment, so the slice's sums are taken per group) and the per-entry
    kernels compute the same normal equations: one sweep each from the same
    start agree to the path's tolerance (the sums only run in another order)."""
    p, X0 = request.getfixturevalue(which)
    out = {}
    for gram in (bfc.GRAM_AUTO, bfc.GRAM_CUDA):
        # group_ratio 2: every middle level on the grouped Gram
        with make(p, prec, gram_impl=gram, group_ratio=2.0) as c:
            assert all(c.level_groups(m)[1] == (gram == bfc.GRAM_AUTO) for m in range(1, p.L + 1))
            c.set_factors(X0)
            st = c.sweep()
            out[gram] = (c.get_factors(), st)
    xa = oracle.eval_entries(p.n, p.L, p.b, p.r, out[bfc.GRAM_AUTO][0], p.it, p.jt)
    xc = oracle.eval_entries(p.n, p.L, p.b, p.r, out[bfc.GRAM_CUDA][0], p.it, p.jt)
    assert rel_dev(xa, xc) <= TOL[prec]
    fa, fc = out[bfc.GRAM_AUTO][1]["objective"], out[bfc.GRAM_CUDA][1]["objective"]
    assert abs(fa - fc) <= TOL[prec] * abs(fc)


@pytest.mark.parametrize("prec", PRECS)
def test_ten_sweeps_cfg1_final_test_error(cfg1, prec):
    p, X0 = cfg1
    Xo = X0
    for _ in range(p.sweeps):
        Xo, _ = oracle_sweep(p, Xo, prec)
    te_o = oracle.rel_err(p.n, p.L, p.b, p.r, Xo, p.it, p.jt, p.tt)
    with make(p, prec) as c:
        c.set_factors(X0)
        hist = [c.sweep() for _ in range(p.sweeps)]
    assert abs(hist[-1]["test_rel_err"] - te_o) <= 1e-4
    objs = [h["objective"] for h in hist]
    assert all(b_ <= a_ * (1 + 1e-6) for a_, b_ in zip(objs[:-1], objs[1:]))


# -------------------------------------------------------------- gradient

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("include_reg", [True, False])
def test_grad_parity(cfg2s, prec, include_reg):
    p, X0 = cfg2s
    go, fo = oracle.grad(p.n, p.L, p.b, p.r, p.lam, X0, p.i, p.j, p.t, include_reg=include_reg)
    with make(p, prec) as c:
        c.set_factors(X0)
        gg, fg = c.grad(include_reg)
    assert abs(fg - fo) <= TOL[prec] * abs(fo)
    scale = np.abs(go).max()
    assert np.abs(gg - go).max() <= TOL[prec] * scale


@pytest.fixture(scope="module", params=[11, 12])
def high_rank(request):
    # ranks 11 and 12 (12 is the rank estimate of the Radon convergence study,
    # Sec. 5.3): D = r^2 = 121 / 144 features per middle-level system.  Data
    # from a planted random butterfly of the same rank, a random start: the
    # block systems are well determined (about 920 entries per slice)
    r = request.param
    n, L, b = 256, 4, 16
    Xt = synth.random_factors(n, L, r, 500 + r)
    X0 = synth.random_factors(n, L, r, 600 + r)
    i, j = synth.draw_pairs(n, 16 * n * 8, 700 + r)
    t = oracle.eval_entries(n, L, b, r, Xt, i, j)
    return (n, L, b, r, 1e-8, i, j, t), X0


@pytest.mark.parametrize("prec", PRECS)
def test_one_sweep_and_gradient_parity_high_rank(high_rank, prec):
    (n, L, b, r, lam, i, j, t), X0 = high_rank
    Xo, st_o = oracle.als_sweep(n, L, b, r, lam, X0, i, j, t, ridge_rel=RIDGE[prec])
    go, fo = oracle.grad(n, L, b, r, lam, X0, i, j, t, include_reg=True)
    with bfc.Completion(n, L, b, r, lam, i, j, t, prec=prec) as c:
        c.set_factors(X0)
        gg, fg = c.grad(True)
        st = c.sweep()
        Xg = c.get_factors()
    tol = TOL[prec]
    assert abs(fg - fo) <= tol * abs(fo)
    assert np.abs(gg - go).max() <= tol * np.abs(go).max()
    # rounding amplified by the worst-conditioned block system (kappa_max
    # about 5e4 / 1.2e5 here: 1e-11 in FP64, 3e-3 / 7e-3 in complex64)
    kappa = max(float(cs.max()) for cs in block_conditions(X0, Xo, i, j, t, n, L, b, r, lam, RIDGE[prec])
                if cs.size)
    tol = max(tol, kappa * (2.0 ** -52 if prec == bfc.PREC_FP64 else 2.0 ** -24))
    assert abs(st["objective"] - st_o["objective"]) <= tol * abs(st_o["objective"])
    assert abs(st["train_rel_err"] - st_o["train_rel_err"]) <= tol * st_o["train_rel_err"]
    xg = oracle.eval_entries(n, L, b, r, Xg, i, j)
    xo = oracle.eval_entries(n, L, b, r, Xo, i, j)
    assert rel_dev(xg, xo) <= tol, (rel_dev(xg, xo), tol, kappa)


# ------------------------------------------------------------ init paths

@pytest.mark.parametrize("prec", PRECS)
def test_lowrank_init_parity(cfg1, prec):
    p, _ = cfg1
    A0, B0 = synth.random_lowrank_start(p, p.r)
    # the low-rank completion runs in the context's precision and reading
    A, B = oracle.lr_complete(p.n, p.r, p.lam, A0, B0, p.i, p.j, p.t, 10, ridge_rel=RIDGE[prec])
    Xo = oracle.embed_lowrank(p.n, p.L, p.b, p.r, A, B)
    with make(p, prec) as c:
        c.lowrank_init(A0, B0, 10)
        Xg = c.get_factors()
    for (ii, jj) in [(p.i, p.j), (p.it, p.jt)]:
        xg = oracle.eval_entries(p.n, p.L, p.b, p.r, Xg, ii, jj)
        xo = oracle.eval_entries(p.n, p.L, p.b, p.r, Xo, ii, jj)
        assert rel_dev(xg, xo) <= TOL[prec]


def test_complete_matches_oracle_workflow(cfg1):
    p, _ = cfg1
    A0, B0 = synth.random_lowrank_start(p, p.r)   # same SplitMix64 recipe as the library's
    A, B = oracle.lr_complete(p.n, p.r, p.lam, A0, B0, p.i, p.j, p.t, 10)
    Xo = oracle.embed_lowrank(p.n, p.L, p.b, p.r, A, B)
    for _ in range(p.sweeps):
        Xo, st_o = oracle.als_sweep(p.n, p.L, p.b, p.r, p.lam, Xo, p.i, p.j, p.t)
    te_o = oracle.rel_err(p.n, p.L, p.b, p.r, Xo, p.it, p.jt, p.tt)
    with make(p, bfc.PREC_FP64, max_sweeps=p.sweeps, tol=0.0, seed=p.seed + synth.SEED_INIT,
              init_kind=1, lr_rank=p.r, lr_sweeps=10) as c:
        hist = c.complete()
    assert len(hist) == p.sweeps
    assert abs(hist[-1]["test_rel_err"] - te_o) <= 1e-6


def test_complete_stops_at_tolerance(cfg1):
    p, X0 = cfg1
    with make(p, bfc.PREC_C64, max_sweeps=30, tol=5e-3) as c:
        c.set_factors(X0)
        hist = c.complete()
    assert hist[-1]["train_rel_err"] < 5e-3
    assert all(h["train_rel_err"] >= 5e-3 for h in hist[:-1])


@pytest.mark.parametrize("prec", PRECS)
def test_graph_replay_equals_direct_launches(cfg2s, prec):
    """bfc_als_sweep replays a captured CUDA graph of the sweep unless kernel
    profiling is on; both paths run the same kernels in the same order, so
    three sweeps from the same start give bit-identical factors, errors and
    launch counts."""
    p, X0 = cfg2s
    out = {}
    for profiled in (True, False):
        with make(p, prec) as c:
            c.set_factors(X0)
            c.profile(profiled)
            hist = [c.sweep() for _ in range(3)]
            out[profiled] = (c.get_factors(), hist)
    (Xd, hd), (Xg, hg) = out[True], out[False]
    assert np.array_equal(Xd.view(np.float64), Xg.view(np.float64))
    for a, b_ in zip(hd, hg):
        assert a["train_rel_err"] == b_["train_rel_err"]
        assert a["test_rel_err"] == b_["test_rel_err"]
        assert a["launches"] == b_["launches"]


# ------------------------------------------------------------ edge cases

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,L,b,r", [(48, 0, 48, 3), (24, 3, 3, 2), (64, 5, 2, 1), (96, 4, 6, 5),
                                     (128, 3, 16, 7)])
def test_odd_shapes_one_sweep(prec, n, L, b, r):
    # leaf sizes that are not powers of two, L = 0 (low-rank), rank 1, ragged
    # and empty slices (few observations)
    X0 = synth.random_factors(n, L, r, 3 + n)
    i, j = synth.draw_pairs(n, min(n * n, 6 * n * max(1, L) + 11), 8 + n)
    t = synth.helmholtz_line(n, math.pi * n / 8, 1.0, i, j)
    lam = 1e-6
    Xo, st_o = oracle.als_sweep(n, L, b, r, lam, X0, i, j, t, ridge_rel=RIDGE[prec])
    with bfc.Completion(n, L, b, r, lam, i, j, t, prec=prec) as c:
        c.set_factors(X0)
        st = c.sweep()
        Xg = c.get_factors()
    tol = TOL[prec]
    if prec == bfc.PREC_C64:
        # complex64 rounding amplified by the worst-conditioned block system
        kappa = max(float(cs.max()) for cs in block_conditions(X0, Xo, i, j, t, n, L, b, r, lam,
                                                                 RIDGE[prec]) if cs.size)
        tol = max(tol, kappa * 2.0 ** -24)
    assert abs(st["objective"] - st_o["objective"]) <= tol * abs(st_o["objective"])
    xg = oracle.eval_entries(n, L, b, r, Xg, i, j)
    xo = oracle.eval_entries(n, L, b, r, Xo, i, j)
    assert rel_dev(xg, xo) <= tol


@pytest.mark.parametrize("prec", PRECS)
def test_singular_fiber_kept_and_counted(prec):
    n, L, b, r = 16, 1, 8, 2
    X0 = synth.random_factors(n, L, r, 3)
    i, j = synth.draw_pairs(n, 200, 5)
    keep = i != 3
    i, j = i[keep], j[keep]
    t = synth.helmholtz_line(n, 10.0, 1.0, i, j)
    _, st_o = oracle.als_sweep(n, L, b, r, 0.0, X0, i, j, t)
    with bfc.Completion(n, L, b, r, 0.0, i, j, t, prec=prec) as c:
        c.set_factors(X0)
        st = c.sweep()
        Xg = c.get_factors()
    assert st["singular_slices"] == st_o["singular"] >= 1
    np.testing.assert_array_equal(Xg[3 * r:4 * r], X0[3 * r:4 * r])


def test_invalid_inputs_rejected():
    n, L, b, r = 64, 2, 16, 2
    i, j = synth.draw_pairs(n, 100, 1)
    t = synth.helmholtz_line(n, 5.0, 1.0, i, j)
    with pytest.raises(bfc.BfcError, match="EINVAL"):
        bfc.Completion(n, L, 8, r, 1e-6, i, j, t)             # n != b 2^L
    with pytest.raises(bfc.BfcError, match="EINVAL"):
        bfc.Completion(n, L, b, 13, 1e-6, i, j, t)            # rank too large (max 12)
    with pytest.raises(bfc.BfcError, match="EINVAL"):
        bfc.Completion(n, L, b, r, -1.0, i, j, t)             # lambda < 0
    bad = i.copy()
    bad[7] = n
    with pytest.raises(bfc.BfcError, match="outside"):
        bfc.Completion(n, L, b, r, 1e-6, bad, j, t)
    dup_i = np.concatenate([i, i[:1]])
    dup_j = np.concatenate([j, j[:1]])
    with pytest.raises(bfc.BfcError, match="duplicate"):
        bfc.Completion(n, L, b, r, 1e-6, dup_i, dup_j, np.concatenate([t, t[:1]]))
    tn = t.copy()
    tn[3] = np.nan
    with pytest.raises(bfc.BfcError, match="NaN"):
        bfc.Completion(n, L, b, r, 1e-6, i, j, tn)
    with bfc.Completion(n, L, b, r, 1e-6, i, j, t) as c:
        with pytest.raises(bfc.BfcError, match="outside"):
            c.eval(np.array([0, -1]), np.array([0, 0]))


# ------------------------------------------------- full size (n = 65536)

@pytest.fixture(scope="module")
def cfg3():
    p = synth.config(3)
    with bfc.Completion(p.n, p.L, p.b, p.r, p.lam, p.i, p.j, p.t, p.it, p.jt, p.tt,
                        prec=bfc.PREC_C64) as c:
        A0, B0 = synth.random_lowrank_start(p, p.r)
        c.lowrank_init(A0, B0, 10)
        X0 = c.get_factors()
        s1 = c.sweep()
        X1 = c.get_factors()
        s2 = c.sweep()
    return p, X0, X1, s1, s2


def test_full_size_orders_are_stable_sorts():
    """Every level order at n = 65536 (3.77 M entries): a stable sort by the
    level key, further by row or column inside the slices of the grouped
    levels, with the oracle's key formula; group counts per level."""
    p = synth.config(3)
    keys = [p.i.astype(np.int64)] + [k.astype(np.int64) for k in level_keys(p.i, p.j, p.L, p.b)] + \
        [p.j.astype(np.int64)]
    with bfc.Completion(p.n, p.L, p.b, p.r, p.lam, p.i, p.j, p.t, prec=bfc.PREC_C64) as c:
        grouped = 0
        for level in range(p.L + 2):
            key = keys[level]
            sub = np.zeros(p.nnz, dtype=np.int64)
            if 1 <= level <= p.L:
                other = (p.j if 2 * level > p.L + 1 else p.i).astype(np.int64)
                ngroups, on = c.level_groups(level)
                assert ngroups == np.unique(key * p.n + other).size
                if on:
                    sub = other
                    grouped += 1
            perm, seg = c.order(level)
            np.testing.assert_array_equal(perm, np.lexsort((sub, key)))
            K = p.n if level in (0, p.L + 1) else 1 << (p.L + 1)
            np.testing.assert_array_equal(seg, np.searchsorted(np.sort(key), np.arange(K + 1)))
        assert grouped == 4   # levels 1, 2, 11 and 12 have fewer than 0.1 groups per entry


def test_full_size_reported_errors_match_oracle(cfg3):
    p, X0, X1, s1, s2 = cfg3
    tr = oracle.rel_err(p.n, p.L, p.b, p.r, X1, p.i, p.j, p.t)
    te = oracle.rel_err(p.n, p.L, p.b, p.r, X1, p.it, p.jt, p.tt)
    assert abs(s1["train_rel_err"] - tr) <= 1e-4 * tr
    assert abs(s1["test_rel_err"] - te) <= 1e-4 * te
    assert s2["objective"] <= s1["objective"] * (1 + 1e-5)
    assert s1["singular_slices"] == 0


def test_full_size_sampled_blocks_are_optimal(cfg3):
    # For sampled slices of every middle level, the GPU's new slice minimizes
    # that slice's regularized least-squares problem (design vectors rebuilt
    # here from the factors before and after the sweep).
    p, X0, X1, s1, s2 = cfg3
    z1o, Zo, zLo = split_packed(X0, p.n, p.L, p.b, p.r)
    z1n, Zn, zLn = split_packed(X1, p.n, p.L, p.b, p.r)
    keys = level_keys(p.i, p.j, p.L, p.b)
    rng = np.random.default_rng(0)
    for m in range(1, p.L + 1):
        for k in rng.choice(1 << (p.L + 1), 2, replace=False):
            sel = np.nonzero(keys[m - 1] == k)[0]
            if sel.size == 0:
                continue
            Zmix = np.concatenate([Zn[: m - 1], Zo[m - 1:]])
            h_new, _ = envs_numpy(z1n, Zmix, zLo, p.i[sel], p.j[sel], p.L, p.b, p.r)
            _, w_o = envs_numpy(z1o, Zo, zLo, p.i[sel], p.j[sel], p.L, p.b, p.r)
            A = np.einsum("ea,ec->eac", h_new[m], w_o[m]).reshape(sel.size, p.r * p.r)
            s_opt = lstsq_block(A, p.t[sel], p.lam)
            f_opt = block_objective(A, p.t[sel], p.lam, s_opt)
            f_gpu = block_objective(A, p.t[sel], p.lam, Zn[m - 1, k].ravel())
            assert f_gpu <= f_opt * (1 + 1e-4) + 1e-12


# ---------------------------------------------------------------- L-BFGS

@pytest.mark.parametrize("prec", PRECS)
def test_lbfgs_parity(cfg2s, prec):
    p, X0 = cfg2s
    iters = 8
    Xo, fo = oracle.lbfgs(p.n, p.L, p.b, p.r, p.lam, X0, p.i, p.j, p.t, iters)
    with make(p, prec) as c:
        c.set_factors(X0)
        hist = c.lbfgs(iters)
        Xg = c.get_factors()
    fg = [h["objective"] for h in hist]
    assert len(fg) == iters
    assert all(b_ <= a_ * (1 + 1e-6) for a_, b_ in zip(fg[:-1], fg[1:]))
    if prec == bfc.PREC_FP64:
        np.testing.assert_allclose(fg, fo, rtol=1e-8)
        assert rel_dev(Xg, Xo) <= 1e-6
    else:
        # complex64 gradients: the trajectory agrees to the complex64 tolerance
        np.testing.assert_allclose(fg, fo, rtol=TOL[prec])


# ------------------------------------- the n = 4096 workload at its own size

@pytest.fixture(scope="module")
def cfg2():
    p = synth.config(2)
    with oracle.threads(oracle.max_threads()):
        return p, lr_start(p)


@pytest.mark.parametrize("prec", PRECS)
def test_cfg2_full_size_one_sweep_parity(cfg2, prec):
    """n = 4096, L = 8, r = 6, 6 n log2 n samples with noise: one sweep from the
    oracle's low-rank start, against the oracle, entries and errors."""
    p, X0 = cfg2
    with oracle.threads(oracle.max_threads()):
        Xo, st_o = oracle_sweep(p, X0, prec)
    with make(p, prec) as c:
        c.set_factors(X0)
        st = c.sweep()
        Xg = c.get_factors()
    tol = TOL[prec]
    assert abs(st["objective"] - st_o["objective"]) <= tol * abs(st_o["objective"])
    assert abs(st["train_rel_err"] - st_o["train_rel_err"]) <= tol * st_o["train_rel_err"]
    with oracle.threads(oracle.max_threads()):
        for (ii, jj) in [(p.i, p.j), (p.it, p.jt)]:
            xg = oracle.eval_entries(p.n, p.L, p.b, p.r, Xg, ii, jj)
            xo = oracle.eval_entries(p.n, p.L, p.b, p.r, Xo, ii, jj)
            assert rel_dev(xg, xo) <= tol


def test_cfg2_full_size_lbfgs_trajectory(cfg2):
    """Config 2's gradient completion (20 L-BFGS iterations, memory 10) at
    n = 4096 in FP64 against the pinned oracle L-BFGS."""
    p, X0 = cfg2
    iters = 20
    with oracle.threads(oracle.max_threads()):
        Xo, fo = oracle.lbfgs(p.n, p.L, p.b, p.r, p.lam, X0, p.i, p.j, p.t, iters)
    with make(p, bfc.PREC_FP64) as c:
        c.set_factors(X0)
        hist = c.lbfgs(iters)
    np.testing.assert_allclose([h["objective"] for h in hist], fo, rtol=1e-8)


@pytest.mark.parametrize("prec", PRECS)
def test_batch_member_one_sweep_parity(prec):
    """A rank-8, n = 16384 member of the 64-problem batched workload: one sweep
    from the oracle's low-rank start against the oracle."""
    p = next(q for q in synth.batch_problems(64) if q.r == 8 and q.n == 16384)
    with oracle.threads(oracle.max_threads()):
        X0 = lr_start(p)
        Xo, st_o = oracle_sweep(p, X0, prec)
    with make(p, prec) as c:
        c.set_factors(X0)
        st = c.sweep()
        Xg = c.get_factors()
    tol = TOL[prec]
    assert abs(st["objective"] - st_o["objective"]) <= tol * abs(st_o["objective"])
    with oracle.threads(oracle.max_threads()):
        xg = oracle.eval_entries(p.n, p.L, p.b, p.r, Xg, p.it, p.jt)
        xo = oracle.eval_entries(p.n, p.L, p.b, p.r, Xo, p.it, p.jt)
    assert rel_dev(xg, xo) <= tol


def test_measured_alu_peaks_are_plausible():
    f32, f64 = bfc.bfc_measure_alu_peaks()
    # FMA-chain rates on a full GPU: tens of TFLOP/s in FP32, FP64 far below it
    assert 5.0 < f32 < 500.0
    assert 0.05 < f64 < f32 / 4
