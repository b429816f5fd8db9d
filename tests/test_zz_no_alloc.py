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
import ctypes

import numpy as np
import pytest

import paper_2510_17734_gb300 as bfc
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10
CAP = 4194304


def _device_inputs(torch, p, X):
    dev = torch.device("cuda", 0)
    F = torch.from_numpy(X.view(np.float64).copy()).to(dev)
    ii = torch.from_numpy(p.i.astype(np.int32)).to(dev)
    jj = torch.from_numpy(p.j.astype(np.int32)).to(dev)
    tt = torch.from_numpy(p.t.astype(np.complex128).view(np.float64).copy()).to(dev)
    return dev, F, ii, jj, tt


def _reference(p, X):
    with bfc.Completion(p.n, p.L, p.b, p.r, p.lam, p.i, p.j, p.t, prec=bfc.PREC_FP64) as c:
        c.set_factors(X)
        _, f_ref = c.grad(include_reg=False)          # 1/2 sum |x - t|^2 over training
    return f_ref, float(np.sum(np.abs(p.t) ** 2))


def _check_sums(torch, sums, f_ref, den_ref, tag):
    torch.cuda.synchronize()
    num, den = sums.cpu().tolist()
    assert abs(0.5 * num - f_ref) <= TOL * abs(f_ref), (tag, 0.5 * num, f_ref)
    assert abs(den - den_ref) <= TOL * den_ref, (tag, den, den_ref)


def test_noalloc_residual_matches_allocating_path():
    torch = pytest.importorskip("torch")
    p = synth.config(1)
    X = synth.random_factors(p.n, p.L, p.r, 42, sigma=0.5)
    f_ref, den_ref = _reference(p, X)
    dev, F, ii, jj, tt = _device_inputs(torch, p, X)
    for call in range(2):
        sums = torch.full((2,), -1.0, dtype=torch.float64, device=dev)
        bfc.bfc_residual_noalloc(p.n, p.L, p.b, p.r, F, ii, jj, tt, sums)
        _check_sums(torch, sums, f_ref, den_ref, call)


def test_noalloc_bad_index_gives_nan_then_recovers():
    """An index outside [0, n) makes both sums NaN; the flag is cleared at the
    start of the next call, which matches the allocating path again."""
    torch = pytest.importorskip("torch")
    p = synth.config(1)
    X = synth.random_factors(p.n, p.L, p.r, 43, sigma=0.5)
    f_ref, den_ref = _reference(p, X)
    dev, F, ii, jj, tt = _device_inputs(torch, p, X)
    bad_i = torch.tensor([p.n], dtype=torch.int32, device=dev)
    bad_j = torch.tensor([0], dtype=torch.int32, device=dev)
    bad_t = torch.zeros(2, dtype=torch.float64, device=dev)
    sums = torch.zeros(2, dtype=torch.float64, device=dev)
    bfc.bfc_residual_noalloc(p.n, p.L, p.b, p.r, F, bad_i, bad_j, bad_t, sums)
    torch.cuda.synchronize()
    assert all(np.isnan(v) for v in sums.cpu().tolist())
    sums = torch.full((2,), -1.0, dtype=torch.float64, device=dev)
    bfc.bfc_residual_noalloc(p.n, p.L, p.b, p.r, F, ii, jj, tt, sums)
    _check_sums(torch, sums, f_ref, den_ref, "after bad index")


def test_noalloc_empty_input_gives_zero_sums():
    torch = pytest.importorskip("torch")
    p = synth.config(1)
    X = synth.random_factors(p.n, p.L, p.r, 44, sigma=0.5)
    dev = torch.device("cuda", 0)
    F = torch.from_numpy(X.view(np.float64).copy()).to(dev)
    e_i = torch.zeros(0, dtype=torch.int32, device=dev)
    e_t = torch.zeros(0, dtype=torch.float64, device=dev)
    sums = torch.full((2,), -1.0, dtype=torch.float64, device=dev)
    bfc.bfc_residual_noalloc(p.n, p.L, p.b, p.r, F, e_i, e_i, e_t, sums)
    torch.cuda.synchronize()
    assert sums.cpu().tolist() == [0.0, 0.0]


def test_noalloc_rejects_oversize_bad_sizes_and_bad_pointers():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    n, L, b, r = 256, 4, 16, 4
    P = bfc.bfc_num_params(n, L, b, r)
    sums = torch.zeros(2, dtype=torch.float64, device=dev)
    F = torch.zeros(2 * P, dtype=torch.float64, device=dev)
    big = torch.zeros(CAP + 1, dtype=torch.int32, device=dev)
    big_t = torch.zeros(2 * (CAP + 1), dtype=torch.float64, device=dev)
    with pytest.raises(bfc.BfcError, match="capacity"):
        bfc.bfc_residual_noalloc(n, L, b, r, F, big, big, big_t, sums)
    del big, big_t
    one = torch.zeros(1, dtype=torch.int32, device=dev)
    t1 = torch.zeros(2, dtype=torch.float64, device=dev)
    with pytest.raises(bfc.BfcError, match="EINVAL"):
        bfc.bfc_residual_noalloc(100, 4, 16, 4, F, one, one, t1, sums)
    # through the C ABI directly (the binding's own checks bypassed): a rank
    # outside [1, 10], a host pointer and a factor vector that is only
    # 8-byte aligned are refused
    lib = bfc.load()
    st = lib.bfc_residual_noalloc(n, L, b, 11, ctypes.c_void_p(F.data_ptr()), 1,
                                  ctypes.c_void_p(one.data_ptr()), ctypes.c_void_p(one.data_ptr()),
                                  ctypes.c_void_p(t1.data_ptr()), ctypes.c_void_p(sums.data_ptr()), None)
    assert st == 1 and "rank" in bfc.bfc_last_error(None)
    host_f = np.zeros(2 * P, dtype=np.float64)
    st = lib.bfc_residual_noalloc(n, L, b, r, host_f.ctypes.data_as(ctypes.c_void_p), 1,
                                  ctypes.c_void_p(one.data_ptr()), ctypes.c_void_p(one.data_ptr()),
                                  ctypes.c_void_p(t1.data_ptr()), ctypes.c_void_p(sums.data_ptr()), None)
    assert st == 1 and "device memory" in bfc.bfc_last_error(None)
    F2 = torch.zeros(2 * P + 1, dtype=torch.float64, device=dev)
    st = lib.bfc_residual_noalloc(n, L, b, r, ctypes.c_void_p(F2.data_ptr() + 8), 1,
                                  ctypes.c_void_p(one.data_ptr()), ctypes.c_void_p(one.data_ptr()),
                                  ctypes.c_void_p(t1.data_ptr()), ctypes.c_void_p(sums.data_ptr()), None)
    assert st == 1 and "aligned" in bfc.bfc_last_error(None)
    # the binding checks device, dtype and lengths before the call
    with pytest.raises(bfc.BfcError, match="CUDA tensor"):
        bfc.bfc_residual_noalloc(n, L, b, r, F.cpu(), one, one, t1, sums)
    with pytest.raises(bfc.BfcError, match="elements"):
        bfc.bfc_residual_noalloc(n, L, b, r, F, one, one, torch.zeros(4, dtype=torch.float64, device=dev), sums)
