"""The allocation-free entry point bfc_residual_noalloc, for callers that
cannot call cudaMalloc (a host application whose memory pool owns the
device, or a caller that cannot accept an allocation at call time).

Its residual sums on caller-owned device buffers must equal what the
allocating path reports for the same factors and entries: the objective
1/2 sum |x - t|^2 of bfc_grad (FP64 context, no regularization term), within
the FP64 tolerance of the other parity tests, on two calls in a row (the
fixed scratch array keeps the previous call's contents).  This file is named
to be collected last.
"""
import numpy as np
import pytest

import paper_2510_17734_gb300 as bfc
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


def test_noalloc_residual_matches_allocating_path():
    torch = pytest.importorskip("torch")
    p = synth.config(1)
    X = synth.random_factors(p.n, p.L, p.r, 42, sigma=0.5)
    with bfc.Completion(p.n, p.L, p.b, p.r, p.lam, p.i, p.j, p.t, prec=bfc.PREC_FP64) as c:
        c.set_factors(X)
        _, f_ref = c.grad(include_reg=False)          # 1/2 sum |x - t|^2 over training
    dev = torch.device("cuda", 0)
    F = torch.from_numpy(X.view(np.float64).copy()).to(dev)
    ii = torch.from_numpy(p.i.astype(np.int32)).to(dev)
    jj = torch.from_numpy(p.j.astype(np.int32)).to(dev)
    tt = torch.from_numpy(p.t.astype(np.complex128).view(np.float64).copy()).to(dev)
    den_ref = float(np.sum(np.abs(p.t) ** 2))
    for call in range(2):
        sums = torch.full((2,), -1.0, dtype=torch.float64, device=dev)
        bfc.bfc_residual_noalloc(p.n, p.L, p.b, p.r, F, ii, jj, tt, sums)
        torch.cuda.synchronize()
        num, den = sums.cpu().tolist()
        assert abs(0.5 * num - f_ref) <= TOL * abs(f_ref), (call, 0.5 * num, f_ref)
        assert abs(den - den_ref) <= TOL * den_ref, (call, den, den_ref)


def test_noalloc_rejects_oversize_and_bad_sizes():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    sums = torch.zeros(2, dtype=torch.float64, device=dev)
    big = torch.zeros(4194305, dtype=torch.int32, device=dev)
    F = torch.zeros(2, dtype=torch.float64, device=dev)
    with pytest.raises(bfc.BfcError, match="capacity"):
        bfc.bfc_residual_noalloc(256, 4, 16, 4, F, big, big, F, sums)
    one = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(bfc.BfcError, match="EINVAL"):
        bfc.bfc_residual_noalloc(100, 4, 16, 4, F, one, one, F, sums)
    with pytest.raises(bfc.BfcError, match="rank"):
        bfc.bfc_residual_noalloc(256, 4, 16, 11, F, one, one, F, sums)
