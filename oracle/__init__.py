"""Complex128 CPU oracle for butterfly tensor completion (arXiv 2510.17734).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The oracle shares no
code with the CUDA library; both only see the same seeded inputs from
``synth``.  The arithmetic lives in ``bfc_oracle.c`` (plain serial C99
``double complex``); this module compiles it with gcc and marshals numpy
arrays through ctypes.

Functions and the passage each follows:
  tree_bits, slice_id      Eq. (indices), Sec. 3.1; psi^{-1} and Eq.
                           (reshaped_tensors), App. A.2
  num_params               Sec. 2.2 memory count with the App. A.2 reshape
  eval_entries             Eq. (BF_tensor_rep)
  rel_err                  Eq. (BF_convergence)
  objective                Eq. (BF_objective) + lambda/2 ||S||^2 (Sec. 4.1.1)
  als_sweep                Alg. 1 (complex normal equations)
  grad                     Eqs. (grad_butterfly_1/_l/_last)
  embed_lowrank            identity embedding of A B^T (stand-in for Alg. 2)
  lr_complete              Alg. 1 with L = 0 (low-rank matrix completion,
                           Sec. 4.2)
  lbfgs                    gradient completion of f by limited-memory BFGS
                           (Nocedal and Wright, Alg. 7.4) over grad()
  matvec                   X(S) V by the definition u_i = sum_j x_ij v_j (the
                           product Eq. (butterfly-mat-vec) forms by
                           contractions)
  set_threads, threads     the threaded variant: OpenMP over independent
                           systems and entries, bit-identical to serial
Modules: first_order (Alg. 3/4 ADAM, Alg. 5 ADF, App. A.3 sweeps), lr2bf
(Alg. 2), gauge (left orthogonalization), mlp (the learned start's network).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libbfc_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libbfc_oracle.so (portable flags,
    no FMA contraction, so x86 and Arm hosts give identical results)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    # OpenMP for the threaded variant (same arithmetic per system; see
    # set_threads); a compiler without it builds the serial oracle
    res = subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True, text=True)
    if res.returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Stats(ctypes.Structure):
    _fields_ = [("train_rel_err", ctypes.c_double),
                ("objective", ctypes.c_double),
                ("singular", ctypes.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
        lib.bfo_tree_bits.argtypes = [i64, i32, i32, vp]
        lib.bfo_tree_bits.restype = None
        lib.bfo_psi_inv.argtypes = [vp, i32]
        lib.bfo_psi_inv.restype = i64
        lib.bfo_slice_id.argtypes = [i64, i64, i32, i32, i32]
        lib.bfo_slice_id.restype = i64
        lib.bfo_num_params.argtypes = [i64, i32, i32, i32]
        lib.bfo_num_params.restype = i64
        lib.bfo_eval.argtypes = [i64, i32, i32, i32, vp, i64, vp, vp, vp]
        lib.bfo_eval.restype = None
        lib.bfo_rel_err.argtypes = [i64, i32, i32, i32, vp, i64, vp, vp, vp]
        lib.bfo_rel_err.restype = dbl
        lib.bfo_objective.argtypes = [i64, i32, i32, i32, dbl, vp, i64, vp, vp, vp]
        lib.bfo_objective.restype = dbl
        lib.bfo_als_sweep.argtypes = [i64, i32, i32, i32, dbl, vp, i64, vp, vp, vp,
                                      ctypes.POINTER(_Stats)]
        lib.bfo_als_sweep.restype = i64
        lib.bfo_als_sweep_ridge.argtypes = [i64, i32, i32, i32, dbl, dbl, vp, i64, vp, vp, vp,
                                            ctypes.POINTER(_Stats)]
        lib.bfo_als_sweep_ridge.restype = i64
        lib.bfo_grad.argtypes = [i64, i32, i32, i32, dbl, i32, vp, i64, vp, vp, vp, vp, vp]
        lib.bfo_grad.restype = None
        lib.bfo_embed_lowrank.argtypes = [i64, i32, i32, i32, i32, vp, vp, vp, vp]
        lib.bfo_embed_lowrank.restype = None
        lib.bfo_matvec.argtypes = [i64, i32, i32, i32, vp, i32, vp, vp]
        lib.bfo_matvec.restype = None
        lib.bfo_set_threads.argtypes = [i32]
        lib.bfo_set_threads.restype = None
        lib.bfo_max_threads.argtypes = []
        lib.bfo_max_threads.restype = i32
        _lib = lib
        return lib


def set_threads(threads: int) -> None:
    """Threads of the oracle's parallel loops (independent systems and
    entries; every sum keeps its serial order, so results are bit-identical
    for any thread count).  1 = serial (the default)."""
    _load().bfo_set_threads(int(threads))


def max_threads() -> int:
    """Threads OpenMP would use by default (1 if built without OpenMP)."""
    return int(_load().bfo_max_threads())


class threads:
    """Context manager: run the oracle on `count` threads inside the block."""

    def __init__(self, count: int):
        self.count = count

    def __enter__(self):
        set_threads(self.count)
        return self

    def __exit__(self, *exc):
        set_threads(1)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_params(n: int, L: int, b: int, r: int) -> int:
    return int(_load().bfo_num_params(n, L, b, r))


def tree_bits(i: int, L: int, b: int) -> list[int]:
    out = np.zeros(L + 1, dtype=np.int32)
    _load().bfo_tree_bits(int(i), L, b, _ptr(out))
    return [int(v) for v in out]


def psi_inv(bits) -> int:
    arr = _i32(bits)
    return int(_load().bfo_psi_inv(_ptr(arr), len(arr)))


def slice_id(i: int, j: int, m: int, L: int, b: int) -> int:
    return int(_load().bfo_slice_id(int(i), int(j), m, L, b))


def eval_entries(n, L, b, r, packed, i, j) -> np.ndarray:
    packed = _c128(packed)
    i, j = _i32(i), _i32(j)
    out = np.zeros(len(i), dtype=np.complex128)
    _load().bfo_eval(n, L, b, r, _ptr(packed), len(i), _ptr(i), _ptr(j), _ptr(out))
    return out


def rel_err(n, L, b, r, packed, i, j, t) -> float:
    packed, t = _c128(packed), _c128(t)
    i, j = _i32(i), _i32(j)
    return float(_load().bfo_rel_err(n, L, b, r, _ptr(packed), len(i), _ptr(i), _ptr(j), _ptr(t)))


def objective(n, L, b, r, lam, packed, i, j, t) -> float:
    packed, t = _c128(packed), _c128(t)
    i, j = _i32(i), _i32(j)
    return float(_load().bfo_objective(n, L, b, r, lam, _ptr(packed), len(i), _ptr(i),
                                       _ptr(j), _ptr(t)))


def als_sweep(n, L, b, r, lam, packed, i, j, t, ridge_rel=0.0):
    """One ALS sweep (Alg. 1).  Returns (new_packed, stats dict).  ridge_rel
    > 0 solves every system with max(lam, ridge_rel * trace(Gram) / dim),
    the regularization the precision form uses."""
    out = _c128(packed).copy()
    t = _c128(t)
    i, j = _i32(i), _i32(j)
    st = _Stats()
    _load().bfo_als_sweep_ridge(n, L, b, r, lam, float(ridge_rel), _ptr(out), len(i), _ptr(i), _ptr(j),
                                _ptr(t), ctypes.byref(st))
    return out, {"train_rel_err": st.train_rel_err, "objective": st.objective,
                 "singular": int(st.singular)}


def grad(n, L, b, r, lam, packed, i, j, t, include_reg=True):
    """Gradient (df/dRe + i df/dIm) and objective."""
    packed, t = _c128(packed), _c128(t)
    i, j = _i32(i), _i32(j)
    g = np.zeros_like(packed)
    obj = ctypes.c_double(0.0)
    _load().bfo_grad(n, L, b, r, lam, int(include_reg), _ptr(packed), len(i), _ptr(i),
                     _ptr(j), _ptr(t), _ptr(g), ctypes.byref(obj))
    return g, float(obj.value)


def embed_lowrank(n, L, b, r, A, B, pad=None):
    """Butterfly factors reproducing A B^T (A, B: n x R, R <= r)."""
    A, B = _c128(A), _c128(B)
    R = A.shape[1]
    if pad is None:
        pad = np.zeros((2 * n, max(r - R, 1)), dtype=np.complex128)
    pad = _c128(pad)
    out = np.zeros(num_params(n, L, b, r), dtype=np.complex128)
    _load().bfo_embed_lowrank(n, L, b, r, R, _ptr(A), _ptr(B), _ptr(pad), _ptr(out))
    return out


def matvec(n, L, b, r, packed, V):
    """U = X(S) V by the definition u_i = sum_j x_ij v_j (V: n or n x nvec
    complex128)."""
    packed = _c128(packed)
    V = _c128(V)
    one = V.ndim == 1
    Vm = np.ascontiguousarray(V.reshape(n, -1))
    U = np.zeros_like(Vm)
    _load().bfo_matvec(n, L, b, r, _ptr(packed), Vm.shape[1], _ptr(Vm), _ptr(U))
    return U.ravel() if one else U


def lr_complete(n, R, lam, A0, B0, i, j, t, sweeps, ridge_rel=0.0):
    """Low-rank matrix completion = Alg. 1 with L = 0 (leaf size n).
    Returns (A, B) with X = A B^T."""
    packed = np.concatenate([_c128(A0).ravel(), _c128(B0).ravel()])
    for _ in range(sweeps):
        packed, _st = als_sweep(n, 0, n, R, lam, packed, i, j, t, ridge_rel=ridge_rel)
    return packed[:n * R].reshape(n, R), packed[n * R:].reshape(n, R)


def lbfgs(n, L, b, r, lam, packed, i, j, t, iters, memory=10, c1=1e-4, trace=None):
    """Limited-memory BFGS on the 2P real parameters (Re, Im interleaved) of
    f = 1/2 sum |x - t|^2 + lambda/2 ||S||^2, gradients from grad().
    Two-loop recursion, H0 = gamma I with gamma = s^T y / y^T y of the newest
    pair; backtracking Armijo line search (c1, halving, <= 30 trials) from
    step 1, or 1/||g|| before the first pair; a pair is kept only if
    s^T y > 1e-12 ||s|| ||y||.  Returns (final packed factors, objectives).
    `trace` (a list) receives per iteration (x, g, d, step, f) before the
    step, for the tests that check the direction against the BFGS matrix."""
    def fg(xr):
        g, f = grad(n, L, b, r, lam, xr.view(np.complex128), i, j, t, include_reg=True)
        return f, g.view(np.float64).copy()

    x = _c128(packed).copy().view(np.float64)
    f, g = fg(x)
    S, Y, rho, hist = [], [], [], []
    for k in range(iters):
        q = g.copy()
        alpha = [0.0] * len(S)
        for idx in range(len(S) - 1, -1, -1):
            alpha[idx] = rho[idx] * float(S[idx] @ q)
            q -= alpha[idx] * Y[idx]
        gamma = float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1]) if S else 1.0
        d = gamma * q
        for idx in range(len(S)):
            beta = rho[idx] * float(Y[idx] @ d)
            d += S[idx] * (alpha[idx] - beta)
        d = -d
        gtd = float(g @ d)
        if not gtd < 0.0:
            d = -g
            gtd = -float(g @ g)
        step = 1.0 / float(np.sqrt(g @ g)) if (not S and k == 0) else 1.0
        for _ in range(30):
            xt = x + step * d
            ft, gt = fg(xt)
            if ft <= f + c1 * step * gtd:
                break
            step *= 0.5
        if trace is not None:
            trace.append((x.copy(), g.copy(), d.copy(), step, f))
        s_, y_ = xt - x, gt - g
        sy = float(s_ @ y_)
        if sy > 1e-12 * float(np.linalg.norm(s_)) * float(np.linalg.norm(y_)):
            S.append(s_)
            Y.append(y_)
            rho.append(1.0 / sy)
            if len(S) > memory:
                S.pop(0), Y.pop(0), rho.pop(0)
        x, g, f = xt, gt, ft
        hist.append(f)
    return x.view(np.complex128).copy(), hist
