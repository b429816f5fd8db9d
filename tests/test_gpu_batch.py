"""Batched form (bfc_batch_complete) and the FP64 refinement sweeps of the
precision form, through the C ABI.

The batch must reproduce, bit for bit, what each problem's own
bfc_complete does with the same parameters when the kernel choice is fixed
(the rounds only reorder independent problems' work across streams); the
autotuned batch must reach the same errors.  The refinement sweeps must equal
FP64 sweeps run from the complex64 result.
"""
import numpy as np
import pytest

import paper_2510_17734_gb300 as bfc
import synth

pytestmark = pytest.mark.gpu


def make(p, prec, **kw):
    return bfc.Completion(p.n, p.L, p.b, p.r, p.lam, p.i, p.j, p.t, p.it, p.jt, p.tt, prec=prec, **kw)


def problems():
    # four small problems of the batched workload (n = 1024 / 2048, r in {4, 6, 8})
    return synth.batch_problems(count=4, n_choices=(1024, 2048))


PRECS = [bfc.PREC_C64, bfc.PREC_FP64, bfc.PREC_C64, bfc.PREC_C64]


def kwargs(q, gram):
    return dict(max_sweeps=6, tol=1e-12, seed=1000 + q, init_kind=1, lr_sweeps=5, gram_impl=gram)


def test_batch_equals_individual_runs_bitwise():
    probs = problems()
    singles = []
    for q, p in enumerate(probs):
        with make(p, PRECS[q], **kwargs(q, bfc.GRAM_CUDA)) as c:
            hist = c.complete()
            singles.append((hist[-1], c.get_factors()))
    batch = [make(p, PRECS[q], **kwargs(q, bfc.GRAM_CUDA)) for q, p in enumerate(probs)]
    try:
        last = bfc.batch_complete(batch)
        for q, c in enumerate(batch):
            st, X = singles[q]
            assert last[q]["sweep"] == st["sweep"] == 6
            np.testing.assert_array_equal(c.get_factors(), X)
            assert last[q]["train_rel_err"] == st["train_rel_err"]
            assert last[q]["launches"] > 0
            # all six sweeps of every problem ran in one graph launch
            assert last[q]["batch_launches"] == 1
    finally:
        for c in batch:
            c.close()


def test_batch_autotuned_reaches_the_same_errors():
    probs = problems()
    ref = []
    for q, p in enumerate(probs):
        with make(p, PRECS[q], **kwargs(q, bfc.GRAM_CUDA)) as c:
            ref.append(c.complete()[-1]["train_rel_err"])
    batch = [make(p, PRECS[q], **kwargs(q, bfc.GRAM_AUTO)) for q, p in enumerate(probs)]
    try:
        last = bfc.batch_complete(batch)
        for q in range(len(probs)):
            assert last[q]["sweep"] == 6
            assert last[q]["batch_launches"] == 1
            assert abs(last[q]["train_rel_err"] - ref[q]) <= 1e-3 * ref[q]
            assert last[q]["gram_impl"] == (-1 if PRECS[q] == bfc.PREC_FP64 else last[q]["gram_impl"])
            assert last[q]["gram_impl"] in ((-1,) if PRECS[q] == bfc.PREC_FP64 else (0, 1))
    finally:
        for c in batch:
            c.close()


def test_batch_stops_each_problem_at_its_tolerance():
    probs = problems()[:2]
    batch = [make(p, bfc.PREC_C64, max_sweeps=12, tol=[0.5, 1e-12][q], seed=7 + q, init_kind=1,
                  lr_sweeps=5) for q, p in enumerate(probs)]
    try:
        last = bfc.batch_complete(batch)
        assert last[0]["train_rel_err"] < 0.5 and last[0]["sweep"] < 12
        assert last[1]["sweep"] == 12
    finally:
        for c in batch:
            c.close()


def test_empty_batch_and_invalid_batches():
    assert bfc.bfc_batch_complete([]) == []
    p = problems()[0]
    with make(p, bfc.PREC_C64) as c:
        with pytest.raises(bfc.BfcError, match="twice"):
            bfc.bfc_batch_complete([c.ctx, c.ctx])
    with pytest.raises(bfc.BfcError, match="null"):
        bfc.bfc_batch_complete([None])


def test_refinement_sweeps_are_fp64_sweeps_from_the_c64_result():
    p = synth.config(2, n_override=1024)
    kw = dict(max_sweeps=4, tol=1e-12, seed=11, init_kind=1, lr_sweeps=5)
    with make(p, bfc.PREC_C64, **kw) as c:
        X64 = None
        hist = c.complete()
        assert len(hist) == 4
        X64 = c.get_factors()
    with make(p, bfc.PREC_C64, refine_sweeps=2, **kw) as c:
        hist = c.complete()
        assert len(hist) == 6 and [h["sweep"] for h in hist] == [1, 2, 3, 4, 5, 6]
        assert [h["gram_impl"] for h in hist[4:]] == [-1, -1]
        Xr = c.get_factors()
    with make(p, bfc.PREC_FP64) as f:
        f.set_factors(X64)
        f.sweep()
        f.sweep()
        Xf = f.get_factors()
    np.testing.assert_array_equal(Xr, Xf)
