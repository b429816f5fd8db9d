"""Error paths driven by host-side failure injection (bfc_inject_fault); no
GPU fault is caused.

Kind 1: the middle-level solve and gradient kernels of the precision form skip
issuing their bulk copies but still wait for them with a short wait limit, so
the bounded waits expire; the kernels then load the data by plain loads and
the call returns BFC_ETIMEOUT.  Kind 2: the device error word is raised from
the host before the status read.  After injection is switched off the same
context gives results that match the oracle again.
"""
import numpy as np
import pytest

import oracle
import paper_2510_17734_gb300 as bfc
import synth
from helpers import rel_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg1():
    p = synth.config(1)
    A, B = synth.random_lowrank_start(p, p.r)
    A, B = oracle.lr_complete(p.n, p.r, p.lam, A, B, p.i, p.j, p.t, 10)
    return p, oracle.embed_lowrank(p.n, p.L, p.b, p.r, A, B)


def _make(p, prec):
    return bfc.Completion(p.n, p.L, p.b, p.r, p.lam, p.i, p.j, p.t, p.it, p.jt, p.tt, prec=prec)


def _sweep_matches_oracle(c, p, X0, tol):
    Xo, st_o = oracle.als_sweep(p.n, p.L, p.b, p.r, p.lam, X0, p.i, p.j, p.t)
    c.set_factors(X0)
    st = c.sweep()
    assert abs(st["objective"] - st_o["objective"]) <= tol * abs(st_o["objective"])


@pytest.mark.parametrize("kind", [1, 2])
def test_sweep_reports_timeout_and_context_stays_usable(cfg1, kind):
    p, X0 = cfg1
    with _make(p, bfc.PREC_C64) as c:
        c.set_factors(X0)
        c.sweep()                                   # a normal sweep first (graph captured)
        bfc.bfc_inject_fault(c.ctx, kind)
        c.set_factors(X0)
        with pytest.raises(bfc.BfcError, match="ETIMEOUT"):
            c.sweep()
        with pytest.raises(bfc.BfcError, match="ETIMEOUT"):
            c.grad(True)
        bfc.bfc_inject_fault(c.ctx, 0)
        _sweep_matches_oracle(c, p, X0, 1e-4)
        c.set_factors(X0)
        g, f = c.grad(True)
    go, fo = oracle.grad(p.n, p.L, p.b, p.r, p.lam, X0, p.i, p.j, p.t, include_reg=True)
    assert abs(f - fo) <= 1e-4 * abs(fo)
    assert np.abs(g - go).max() <= 1e-3 * np.abs(go).max()


def test_skipped_copies_fall_back_to_plain_loads(cfg1):
    """With kind 1 the kernels finish the work by plain loads: the sweep's
    factors equal those of a sweep without injection (the call still reports
    the expired wait)."""
    p, X0 = cfg1
    with _make(p, bfc.PREC_C64) as c:
        c.profile(True)                             # direct launches: same kernels either way
        c.set_factors(X0)
        c.sweep()
        X_ref = c.get_factors()
        bfc.bfc_inject_fault(c.ctx, 1)
        c.set_factors(X0)
        with pytest.raises(bfc.BfcError, match="ETIMEOUT"):
            c.sweep()
        X_inj = c.get_factors()
        bfc.bfc_inject_fault(c.ctx, 0)
    assert rel_dev(X_inj, X_ref) <= 1e-6


def test_fp64_path_has_no_bulk_copies_but_reports_host_injection(cfg1):
    p, X0 = cfg1
    with _make(p, bfc.PREC_FP64) as c:
        bfc.bfc_inject_fault(c.ctx, 1)              # nothing to skip in FP64
        _sweep_matches_oracle(c, p, X0, 1e-10)
        bfc.bfc_inject_fault(c.ctx, 2)
        with pytest.raises(bfc.BfcError, match="ETIMEOUT"):
            c.sweep()
        bfc.bfc_inject_fault(c.ctx, 0)
        _sweep_matches_oracle(c, p, X0, 1e-10)


def test_inject_rejects_unknown_kind(cfg1):
    p, _ = cfg1
    with _make(p, bfc.PREC_FP64) as c:
        with pytest.raises(bfc.BfcError, match="EINVAL"):
            bfc.bfc_inject_fault(c.ctx, 3)


def test_batch_launch_reports_timeout_and_recovers():
    """An expired bounded wait inside the one-launch batch stops that
    problem's loop on the device; the batch returns BFC_ETIMEOUT and, with
    injection off, the same contexts complete normally."""
    probs = synth.batch_problems(count=2, n_choices=(1024,))
    cs = [bfc.Completion(p.n, p.L, p.b, p.r, p.lam, p.i, p.j, p.t, p.it, p.jt, p.tt, prec=bfc.PREC_C64,
                         max_sweeps=4, tol=1e-12, seed=5 + q, init_kind=1, lr_sweeps=5, gram_impl=bfc.GRAM_CUDA)
          for q, p in enumerate(probs)]
    try:
        bfc.bfc_inject_fault(cs[1].ctx, 1)
        with pytest.raises(bfc.BfcError, match="ETIMEOUT"):
            bfc.batch_complete(cs)
        bfc.bfc_inject_fault(cs[1].ctx, 0)
        last = bfc.batch_complete(cs)
        assert all(st["sweep"] > 0 and np.isfinite(st["train_rel_err"]) for st in last)
        assert all(st["batch_launches"] == 1 for st in last)
    finally:
        for c in cs:
            c.close()
