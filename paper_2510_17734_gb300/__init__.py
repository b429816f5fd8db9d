"""Python binding of libbfc, the GB300 butterfly tensor completion library.

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI declared in include/bfc.h.  The functions below keep
the C names (bfc_create, bfc_als_sweep, ...).  Host data are numpy arrays;
with ``values_on_device=1`` the data arguments are torch CUDA tensors (their
device pointers are passed through).

The library is built in-tree by ``paper_2510_17734_gb300.build`` (or
``__graft_entry__.build()``); loading fails loudly when it is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = [
    "BfcError", "Params", "SweepStats", "KernelProfile", "Completion", "PREC_FP64", "PREC_C64",
    "load", "library_path", "exported_symbols",
    "bfc_num_params", "bfc_create", "bfc_set_stream", "bfc_set_factors", "bfc_get_factors",
    "bfc_eval", "bfc_als_sweep", "bfc_grad", "bfc_lowrank_init", "bfc_complete",
    "bfc_profile_enable", "bfc_profile_read", "bfc_last_error", "bfc_destroy",
    "bfc_decode", "bfc_get_order", "bfc_residual_noalloc", "bfc_lbfgs", "bfc_batch_complete",
    "batch_complete", "GRAM_AUTO", "GRAM_TENSOR", "GRAM_CUDA",
    "bfc_mlp_create", "bfc_mlp_dims", "bfc_mlp_num_params", "bfc_mlp_get_params", "bfc_mlp_set_params",
    "bfc_mlp_set_scaling", "bfc_mlp_forward", "bfc_mlp_grad", "bfc_mlp_train", "bfc_mlp_destroy",
    "bfc_init_learned", "bfc_canonicalize", "Mlp", "bfc_measure_alu_peaks", "bfc_inject_fault",
    "bfc_adam", "bfc_adf", "bfc_matvec", "bfc_lowrank_to_butterfly", "bfc_level_groups",
]

PREC_FP64 = 0
PREC_C64 = 1
GRAM_AUTO = 0     # per middle level: grouped CUDA-core Gram where few row / column groups, else tcgen05 (r <= 8)
GRAM_CUDA = 1     # CUDA-core Gram per entry always
GRAM_TENSOR = 2   # tcgen05 Gram per entry for r <= 8 in the precision form, no grouping
STATUS = {0: "BFC_OK", 1: "BFC_EINVAL", 2: "BFC_ENOMEM", 3: "BFC_ECUDA", 4: "BFC_ESINGULAR",
          5: "BFC_ETIMEOUT", 6: "BFC_ENONFINITE"}

# Every entry point declared in include/bfc.h.
exported_symbols = (
    "bfc_num_params", "bfc_create", "bfc_set_stream", "bfc_set_factors", "bfc_get_factors",
    "bfc_eval", "bfc_als_sweep", "bfc_grad", "bfc_lbfgs", "bfc_lowrank_init", "bfc_complete",
    "bfc_batch_complete", "bfc_decode", "bfc_get_order", "bfc_residual_noalloc",
    "bfc_mlp_create", "bfc_mlp_dims", "bfc_mlp_num_params", "bfc_mlp_get_params", "bfc_mlp_set_params",
    "bfc_mlp_set_scaling", "bfc_mlp_forward", "bfc_mlp_grad", "bfc_mlp_train", "bfc_mlp_destroy",
    "bfc_init_learned", "bfc_canonicalize", "bfc_measure_alu_peaks", "bfc_inject_fault",
    "bfc_adam", "bfc_adf", "bfc_matvec", "bfc_lowrank_to_butterfly", "bfc_level_groups",
    "bfc_profile_enable", "bfc_profile_read", "bfc_last_error", "bfc_destroy",
)


class BfcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("L", ctypes.c_int32), ("b", ctypes.c_int32),
                ("r", ctypes.c_int32), ("lam", ctypes.c_double), ("prec", ctypes.c_int32),
                ("max_sweeps", ctypes.c_int32), ("tol", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("init_kind", ctypes.c_int32), ("lr_rank", ctypes.c_int32),
                ("lr_sweeps", ctypes.c_int32), ("values_on_device", ctypes.c_int32),
                ("refine_sweeps", ctypes.c_int32), ("ridge_rel", ctypes.c_double),
                ("gram_impl", ctypes.c_int32), ("lr2bf_oversample", ctypes.c_int32),
                ("group_ratio", ctypes.c_double)]


class SweepStats(ctypes.Structure):
    _fields_ = [("sweep", ctypes.c_int32), ("train_rel_err", ctypes.c_double),
                ("test_rel_err", ctypes.c_double), ("objective", ctypes.c_double),
                ("sweep_ms", ctypes.c_double), ("entries_per_s", ctypes.c_double),
                ("singular_slices", ctypes.c_int64), ("refined_fallbacks", ctypes.c_int64),
                ("refine_steps", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("gram_impl", ctypes.c_int32), ("batch_launches", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class KernelProfile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load():
    """Load libbfc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libbfc.so is not built ({path}); run "
                               "`python -m paper_2510_17734_gb300.build` first")
        lib = ctypes.CDLL(path)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        pp = ctypes.POINTER(Params)
        sp = ctypes.POINTER(SweepStats)
        lib.bfc_num_params.argtypes = [i64, i32, i32, i32]
        lib.bfc_num_params.restype = i64
        lib.bfc_create.argtypes = [pp, i64, vp, vp, vp, i64, vp, vp, vp, ctypes.POINTER(vp)]
        lib.bfc_create.restype = i32
        lib.bfc_set_stream.argtypes = [vp, vp]
        lib.bfc_set_stream.restype = i32
        lib.bfc_set_factors.argtypes = [vp, vp]
        lib.bfc_set_factors.restype = i32
        lib.bfc_get_factors.argtypes = [vp, vp]
        lib.bfc_get_factors.restype = i32
        lib.bfc_eval.argtypes = [vp, i64, vp, vp, vp]
        lib.bfc_eval.restype = i32
        lib.bfc_als_sweep.argtypes = [vp, sp]
        lib.bfc_als_sweep.restype = i32
        lib.bfc_grad.argtypes = [vp, i32, vp, ctypes.POINTER(dbl)]
        lib.bfc_grad.restype = i32
        lib.bfc_lbfgs.argtypes = [vp, i32, i32, sp, i32, ctypes.POINTER(i32)]
        lib.bfc_lbfgs.restype = i32
        lib.bfc_lowrank_init.argtypes = [vp, i32, i32, vp, vp]
        lib.bfc_lowrank_init.restype = i32
        lib.bfc_complete.argtypes = [vp, sp, i32, ctypes.POINTER(i32)]
        lib.bfc_complete.restype = i32
        lib.bfc_batch_complete.argtypes = [i32, ctypes.POINTER(vp), sp]
        lib.bfc_batch_complete.restype = i32
        u64 = ctypes.c_uint64
        lib.bfc_mlp_create.argtypes = [i32, i32, i64, u64, ctypes.POINTER(vp)]
        lib.bfc_mlp_create.restype = i32
        lib.bfc_mlp_dims.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i64)]
        lib.bfc_mlp_dims.restype = None
        lib.bfc_mlp_num_params.argtypes = [vp]
        lib.bfc_mlp_num_params.restype = i64
        lib.bfc_mlp_get_params.argtypes = [vp, vp]
        lib.bfc_mlp_get_params.restype = i32
        lib.bfc_mlp_set_params.argtypes = [vp, vp]
        lib.bfc_mlp_set_params.restype = i32
        lib.bfc_mlp_set_scaling.argtypes = [vp, vp, vp, vp, vp]
        lib.bfc_mlp_set_scaling.restype = i32
        lib.bfc_mlp_forward.argtypes = [vp, i32, vp, vp]
        lib.bfc_mlp_forward.restype = i32
        lib.bfc_mlp_grad.argtypes = [vp, i32, vp, vp, vp, ctypes.POINTER(dbl)]
        lib.bfc_mlp_grad.restype = i32
        lib.bfc_mlp_train.argtypes = [vp, i32, vp, vp, i32, i32, dbl, u64, vp]
        lib.bfc_mlp_train.restype = i32
        lib.bfc_mlp_destroy.argtypes = [vp]
        lib.bfc_mlp_destroy.restype = None
        lib.bfc_init_learned.argtypes = [vp, vp, dbl, dbl, i32, ctypes.POINTER(i32), ctypes.POINTER(dbl)]
        lib.bfc_init_learned.restype = i32
        lib.bfc_canonicalize.argtypes = [vp]
        lib.bfc_canonicalize.restype = i32
        lib.bfc_measure_alu_peaks.argtypes = [ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
        lib.bfc_measure_alu_peaks.restype = i32
        lib.bfc_decode.argtypes = [i64, i32, i32, i64, vp, vp, vp]
        lib.bfc_decode.restype = i32
        lib.bfc_get_order.argtypes = [vp, i32, vp, vp]
        lib.bfc_get_order.restype = i32
        lib.bfc_level_groups.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(i32)]
        lib.bfc_level_groups.restype = i32
        lib.bfc_residual_noalloc.argtypes = [i64, i32, i32, i32, vp, i64, vp, vp, vp, vp, vp]
        lib.bfc_residual_noalloc.restype = i32
        lib.bfc_adam.argtypes = [vp, i32, dbl, dbl, dbl, dbl, sp, i32, ctypes.POINTER(i32)]
        lib.bfc_adam.restype = i32
        lib.bfc_adf.argtypes = [vp, i32, sp, i32, ctypes.POINTER(i32)]
        lib.bfc_adf.restype = i32
        lib.bfc_matvec.argtypes = [vp, i32, vp, vp]
        lib.bfc_matvec.restype = i32
        lib.bfc_lowrank_to_butterfly.argtypes = [vp, i32, vp, vp, i32, vp]
        lib.bfc_lowrank_to_butterfly.restype = i32
        lib.bfc_inject_fault.argtypes = [vp, i32]
        lib.bfc_inject_fault.restype = i32
        lib.bfc_profile_enable.argtypes = [vp, i32]
        lib.bfc_profile_enable.restype = i32
        lib.bfc_profile_read.argtypes = [vp, ctypes.POINTER(KernelProfile), i32, ctypes.POINTER(i32)]
        lib.bfc_profile_read.restype = i32
        lib.bfc_last_error.argtypes = [vp]
        lib.bfc_last_error.restype = ctypes.c_char_p
        lib.bfc_destroy.argtypes = [vp]
        lib.bfc_destroy.restype = None
        _lib = lib
        return lib


# ------------------------------------------------------------ marshalling

def _ptr(a):
    """Data pointer of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _host_i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def _host_c128(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.complex128)


def _check(status, ctx=None):
    if status != 0:
        msg = load().bfc_last_error(ctx).decode(errors="replace")
        raise BfcError(status, msg)


# --------------------------------------------------------- C-named calls

def bfc_num_params(n: int, L: int, b: int, r: int) -> int:
    return int(load().bfc_num_params(n, L, b, r))


def bfc_create(params: Params, i, j, t, it=None, jt=None, tt=None):
    """Returns an opaque context handle (ctypes.c_void_p)."""
    lib = load()
    if not params.values_on_device:
        i, j, t = _host_i32(i), _host_i32(j), _host_c128(t)
        it, jt, tt = _host_i32(it), _host_i32(jt), _host_c128(tt)
    nnz = int(i.shape[0])
    ntest = 0 if it is None else int(it.shape[0])
    out = ctypes.c_void_p()
    st = lib.bfc_create(ctypes.byref(params), nnz, _ptr(i), _ptr(j), _ptr(t), ntest, _ptr(it),
                        _ptr(jt), _ptr(tt), ctypes.byref(out))
    _check(st, None)
    return out


def bfc_set_stream(ctx, stream_handle: int | None):
    _check(load().bfc_set_stream(ctx, ctypes.c_void_p(stream_handle or 0)), ctx)


def bfc_set_factors(ctx, packed):
    _check(load().bfc_set_factors(ctx, _ptr(packed)), ctx)


def bfc_get_factors(ctx, out):
    _check(load().bfc_get_factors(ctx, _ptr(out)), ctx)


def bfc_eval(ctx, i, j, out):
    m = int(i.shape[0])
    _check(load().bfc_eval(ctx, m, _ptr(i), _ptr(j), _ptr(out)), ctx)


def bfc_als_sweep(ctx) -> SweepStats:
    st = SweepStats()
    _check(load().bfc_als_sweep(ctx, ctypes.byref(st)), ctx)
    return st


def bfc_grad(ctx, include_reg: bool, grad_out=None) -> float:
    obj = ctypes.c_double(0.0)
    _check(load().bfc_grad(ctx, int(include_reg), _ptr(grad_out), ctypes.byref(obj)), ctx)
    return float(obj.value)


def bfc_lbfgs(ctx, iters: int, memory: int = 10):
    hist = (SweepStats * max(iters, 1))()
    done = ctypes.c_int32(0)
    _check(load().bfc_lbfgs(ctx, iters, memory, hist, iters, ctypes.byref(done)), ctx)
    return [hist[q] for q in range(done.value)]


def bfc_adam(ctx, iters: int, alpha: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
             sigma: float = 1e-8):
    hist = (SweepStats * max(iters, 1))()
    done = ctypes.c_int32(0)
    _check(load().bfc_adam(ctx, iters, alpha, beta1, beta2, sigma, hist, iters, ctypes.byref(done)), ctx)
    return [hist[q] for q in range(done.value)]


def bfc_adf(ctx, iters: int):
    hist = (SweepStats * max(iters, 1))()
    done = ctypes.c_int32(0)
    _check(load().bfc_adf(ctx, iters, hist, iters, ctypes.byref(done)), ctx)
    return [hist[q] for q in range(done.value)]


def bfc_matvec(ctx, nvec: int, V, U):
    _check(load().bfc_matvec(ctx, nvec, _ptr(V), _ptr(U)), ctx)


def bfc_lowrank_to_butterfly(ctx, R: int, A, B, p: int, gaussians):
    _check(load().bfc_lowrank_to_butterfly(ctx, R, _ptr(A), _ptr(B), p, _ptr(gaussians)), ctx)


def bfc_lowrank_init(ctx, R: int, sweeps: int, A0, B0):
    _check(load().bfc_lowrank_init(ctx, R, sweeps, _ptr(A0), _ptr(B0)), ctx)


def bfc_complete(ctx, history_cap: int = 256):
    hist = (SweepStats * max(history_cap, 1))()
    ns = ctypes.c_int32(0)
    _check(load().bfc_complete(ctx, hist, history_cap, ctypes.byref(ns)), ctx)
    return [hist[q] for q in range(min(ns.value, history_cap))]


def bfc_batch_complete(ctxs):
    """Batched full workflow over independent contexts; returns the last
    sweep's statistics of each."""
    count = len(ctxs)
    arr = (ctypes.c_void_p * max(count, 1))(*[c for c in ctxs])
    last = (SweepStats * max(count, 1))()
    _check(load().bfc_batch_complete(count, arr, last), None)
    return [last[q] for q in range(count)]


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def bfc_mlp_create(in_dim: int, hidden: int, out_dim: int, seed: int = 0):
    out = ctypes.c_void_p()
    _check(load().bfc_mlp_create(in_dim, hidden, out_dim, seed, ctypes.byref(out)), None)
    return out.value


def bfc_mlp_dims(m):
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    load().bfc_mlp_dims(m, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return a.value, b.value, c.value


def bfc_mlp_num_params(m) -> int:
    return int(load().bfc_mlp_num_params(m))


def bfc_mlp_get_params(m):
    out = np.zeros(bfc_mlp_num_params(m), dtype=np.float64)
    _check(load().bfc_mlp_get_params(m, _ptr(out)), None)
    return out


def bfc_mlp_set_params(m, params):
    params = _f64(params)
    _check(load().bfc_mlp_set_params(m, _ptr(params)), None)


def bfc_mlp_set_scaling(m, in_lo, in_hi, out_mean, out_std):
    a, b, c, d = _f64(in_lo), _f64(in_hi), _f64(out_mean), _f64(out_std)
    _check(load().bfc_mlp_set_scaling(m, _ptr(a), _ptr(b), _ptr(c), _ptr(d)), None)


def bfc_mlp_forward(m, x):
    x = _f64(x)
    _, _, out_dim = bfc_mlp_dims(m)
    y = np.zeros((x.shape[0], out_dim), dtype=np.float64)
    _check(load().bfc_mlp_forward(m, x.shape[0], _ptr(x), _ptr(y)), None)
    return y


def bfc_mlp_grad(m, x, y):
    x, y = _f64(x), _f64(y)
    g = np.zeros(bfc_mlp_num_params(m), dtype=np.float64)
    loss = ctypes.c_double(0.0)
    _check(load().bfc_mlp_grad(m, x.shape[0], _ptr(x), _ptr(y), _ptr(g), ctypes.byref(loss)), None)
    return g, float(loss.value)


def bfc_mlp_train(m, x, y, epochs: int, batch: int = 32, lr: float = 1e-3, seed: int = 0):
    x, y = _f64(x), _f64(y)
    hist = np.zeros(max(epochs, 1), dtype=np.float64)
    _check(load().bfc_mlp_train(m, x.shape[0], _ptr(x), _ptr(y), epochs, batch, lr, seed, _ptr(hist)), None)
    return hist[:epochs]


def bfc_mlp_destroy(m):
    load().bfc_mlp_destroy(m)


def bfc_measure_alu_peaks():
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().bfc_measure_alu_peaks(ctypes.byref(a), ctypes.byref(b)), None)
    return float(a.value), float(b.value)


def bfc_canonicalize(ctx):
    _check(load().bfc_canonicalize(ctx), ctx)


def bfc_init_learned(ctx, m, omega: float, offset: float, allow_fallback: bool = True):
    used = ctypes.c_int32(0)
    err = ctypes.c_double(0.0)
    _check(load().bfc_init_learned(ctx, m, omega, offset, int(allow_fallback), ctypes.byref(used),
                                   ctypes.byref(err)), ctx)
    return bool(used.value), float(err.value)


class Mlp:
    """Owner of a bfc_mlp handle (closes on exit)."""

    def __init__(self, in_dim, hidden, out_dim, seed=0):
        self.h = bfc_mlp_create(in_dim, hidden, out_dim, seed)

    def close(self):
        if self.h:
            bfc_mlp_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_complete(completions):
    """bfc_batch_complete over Completion objects; returns stats dicts."""
    return [st.as_dict() for st in bfc_batch_complete([c.ctx for c in completions])]


def bfc_decode(n: int, L: int, b: int, i, j):
    """Level keys (m x (L+2) int32) computed on the GPU."""
    i, j = _host_i32(i), _host_i32(j)
    keys = np.zeros((i.shape[0], L + 2), dtype=np.int32)
    _check(load().bfc_decode(n, L, b, i.shape[0], _ptr(i), _ptr(j), _ptr(keys)), None)
    return keys


def bfc_get_order(ctx, level: int, N: int, K: int):
    perm = np.zeros(N, dtype=np.int32)
    seg = np.zeros(K + 1, dtype=np.int32)
    _check(load().bfc_get_order(ctx, level, _ptr(perm), _ptr(seg)), ctx)
    return perm, seg


def bfc_level_groups(ctx, level: int):
    ng = ctypes.c_int64(0)
    gr = ctypes.c_int32(0)
    _check(load().bfc_level_groups(ctx, level, ctypes.byref(ng), ctypes.byref(gr)), ctx)
    return int(ng.value), bool(gr.value)


def _check_cuda_tensor(x, what, dtype_name, numel=None, min_numel=None):
    if not hasattr(x, "is_cuda") or not x.is_cuda:
        raise BfcError(1, f"{what} must be a CUDA tensor")
    if str(x.dtype) != "torch." + dtype_name:
        raise BfcError(1, f"{what} must have dtype {dtype_name}, not {x.dtype}")
    if not x.is_contiguous():
        raise BfcError(1, f"{what} must be contiguous")
    if numel is not None and x.numel() != numel:
        raise BfcError(1, f"{what} has {x.numel()} elements, expected {numel}")
    if min_numel is not None and x.numel() < min_numel:
        raise BfcError(1, f"{what} has {x.numel()} elements, expected at least {min_numel}")


def bfc_residual_noalloc(n: int, L: int, b: int, r: int, factors, i, j, t, sums, stream=None):
    """Allocation-free residual sums on caller-owned device buffers (torch
    CUDA tensors): sums[0] = sum |t - x|^2, sums[1] = sum |t|^2.  Enqueued on
    `stream` (a raw cudaStream_t handle, None = default stream); no wait.
    factors: float64, 2 * bfc_num_params values; i, j: int32, m each; t:
    float64, 2 m values; sums: float64, at least 2 values."""
    m = int(i.shape[0])
    _check_cuda_tensor(i, "i", "int32")
    _check_cuda_tensor(j, "j", "int32", numel=m)
    _check_cuda_tensor(t, "t", "float64", numel=2 * m)
    _check_cuda_tensor(sums, "sums", "float64", min_numel=2)
    P = bfc_num_params(n, L, b, r)
    if P > 0:
        _check_cuda_tensor(factors, "factors", "float64", numel=2 * P)
    _check(load().bfc_residual_noalloc(n, L, b, r, _ptr(factors), m, _ptr(i), _ptr(j), _ptr(t),
                                       _ptr(sums), ctypes.c_void_p(stream or 0)), None)


def bfc_inject_fault(ctx, kind: int):
    """Test-only failure injection (0 off, 1 skipped bulk copies with expiring
    bounded waits, 2 device error word raised from the host)."""
    _check(load().bfc_inject_fault(ctx, int(kind)), ctx)


def bfc_profile_enable(ctx, enable: bool):
    _check(load().bfc_profile_enable(ctx, int(enable)), ctx)


def bfc_profile_read(ctx, cap: int = 64) -> dict:
    recs = (KernelProfile * cap)()
    cnt = ctypes.c_int32(0)
    _check(load().bfc_profile_read(ctx, recs, cap, ctypes.byref(cnt)), ctx)
    return {recs[q].name.decode(): (int(recs[q].launches), float(recs[q].total_ms))
            for q in range(min(cnt.value, cap))}


def bfc_last_error(ctx=None) -> str:
    return load().bfc_last_error(ctx).decode(errors="replace")


def bfc_destroy(ctx):
    if ctx:
        load().bfc_destroy(ctx)


# ------------------------------------------------------ convenience class

class Completion:
    """Owns one bfc context for host (numpy) data."""

    def __init__(self, n, L, b, r, lam, i, j, t, it=None, jt=None, tt=None, prec=PREC_FP64,
                 max_sweeps=20, tol=1e-3, seed=0, init_kind=0, lr_rank=0, lr_sweeps=10,
                 refine_sweeps=0, ridge_rel=0.0, gram_impl=GRAM_AUTO, lr2bf_oversample=0, group_ratio=0.0):
        self.n, self.L, self.b, self.r = int(n), int(L), int(b), int(r)
        self.params = Params(n=n, L=L, b=b, r=r, lam=lam, prec=prec, max_sweeps=max_sweeps, tol=tol,
                             seed=seed, init_kind=init_kind, lr_rank=lr_rank, lr_sweeps=lr_sweeps,
                             values_on_device=0, refine_sweeps=refine_sweeps, ridge_rel=ridge_rel,
                             gram_impl=gram_impl, lr2bf_oversample=lr2bf_oversample,
                             group_ratio=group_ratio)
        self.P = bfc_num_params(n, L, b, r)
        self._nnz = len(i)
        self.ctx = bfc_create(self.params, i, j, t, it, jt, tt)

    def set_factors(self, packed):
        bfc_set_factors(self.ctx, _host_c128(packed))

    def get_factors(self):
        out = np.zeros(self.P, dtype=np.complex128)
        bfc_get_factors(self.ctx, out)
        return out

    def eval(self, i, j):
        i, j = _host_i32(i), _host_i32(j)
        out = np.zeros(i.shape[0], dtype=np.complex128)
        bfc_eval(self.ctx, i, j, out)
        return out

    def sweep(self) -> dict:
        return bfc_als_sweep(self.ctx).as_dict()

    def grad(self, include_reg=True):
        g = np.zeros(self.P, dtype=np.complex128)
        f = bfc_grad(self.ctx, include_reg, g)
        return g, f

    def lbfgs(self, iters, memory=10):
        return [h.as_dict() for h in bfc_lbfgs(self.ctx, iters, memory)]

    def adam(self, iters, alpha=1e-3, beta1=0.9, beta2=0.999, sigma=1e-8):
        return [h.as_dict() for h in bfc_adam(self.ctx, iters, alpha, beta1, beta2, sigma)]

    def adf(self, iters):
        return [h.as_dict() for h in bfc_adf(self.ctx, iters)]

    def matvec(self, V):
        """X(S) V for V of shape (n,) or (n, nvec), complex128."""
        V = _host_c128(V)
        one = V.ndim == 1
        Vm = np.ascontiguousarray(V.reshape(self.n, -1))
        U = np.zeros_like(Vm)
        bfc_matvec(self.ctx, Vm.shape[1], Vm, U)
        return U.ravel() if one else U

    def lowrank_init(self, A0, B0, sweeps):
        A0, B0 = _host_c128(A0), _host_c128(B0)
        bfc_lowrank_init(self.ctx, A0.shape[1], sweeps, A0, B0)

    def lowrank_to_butterfly(self, A, B, p, gaussians):
        A, B, G = _host_c128(A), _host_c128(B), _host_c128(gaussians)
        bfc_lowrank_to_butterfly(self.ctx, A.shape[1], A, B, p, G)

    def order(self, level):
        N = int(self._nnz)
        K = self.n if level in (0, self.L + 1) else (1 << (self.L + 1))
        return bfc_get_order(self.ctx, level, N, K)

    def level_groups(self, level):
        """(groups, grouped) of a middle level (bfc_level_groups)."""
        return bfc_level_groups(self.ctx, level)

    def canonicalize(self):
        bfc_canonicalize(self.ctx)

    def complete(self, history_cap=256):
        return [h.as_dict() for h in bfc_complete(self.ctx, history_cap)]

    def profile(self, enable=True):
        bfc_profile_enable(self.ctx, enable)

    def profile_read(self):
        return bfc_profile_read(self.ctx)

    def close(self):
        if self.ctx:
            bfc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
