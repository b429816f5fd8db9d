"""Float64 oracle of the learned initializer's network (test infrastructure).

Only the test suite and the bench's CPU leg use it; it shares no code with
the CUDA library.  The network is in -> hidden -> hidden -> out with GELU
(x Phi(x), Phi the standard normal distribution function) after both hidden
layers and a linear output, loss = mean squared error over all outputs of a
batch.  Parameters use the flat layout [W1 | b1 | W2 | b2 | W3 | b3], each W
input-major (W[k][n] at k * fan_out + n).  The CUDA kernels use the weights
rounded to bfloat16; `bf16=True` applies the same rounding here (round to
nearest, ties to even, on the float32 value), everything else is float64.

Backpropagation is written out layer by layer (chain rule); it is pinned by
central finite differences in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import math

import numpy as np


def bf16_round(x):
    """Round to the nearest bfloat16 (8 significant bits), ties to even,
    through the float32 value."""
    f = np.asarray(x, dtype=np.float32).copy()
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16) << 16
    return (rounded & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)


def layout(in_dim, hidden, out_dim):
    sizes = [("W1", in_dim * hidden), ("b1", hidden), ("W2", hidden * hidden), ("b2", hidden),
             ("W3", hidden * out_dim), ("b3", out_dim)]
    off, out = 0, {}
    for name, n in sizes:
        out[name] = (off, n)
        off += n
    return out, off


def unpack(params, in_dim, hidden, out_dim, bf16=True):
    lay, _ = layout(in_dim, hidden, out_dim)
    p = np.asarray(params, dtype=np.float64)
    get = lambda name: p[lay[name][0]:lay[name][0] + lay[name][1]]
    rw = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    W1 = rw(get("W1")).reshape(in_dim, hidden)
    W2 = rw(get("W2")).reshape(hidden, hidden)
    W3 = rw(get("W3")).reshape(hidden, out_dim)
    return W1, get("b1"), W2, get("b2"), W3, get("b3")


_erf = np.vectorize(math.erf)


def gelu(a):
    return 0.5 * a * (1.0 + _erf(a / math.sqrt(2.0)))


def gelu_grad(a):
    cdf = 0.5 * (1.0 + _erf(a / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * a * a) / math.sqrt(2.0 * math.pi)
    return cdf + a * pdf


def forward(params, dims, x, bf16=True):
    """Outputs (batch x out) for normalized inputs x (batch x in)."""
    in_dim, hidden, out_dim = dims
    W1, b1, W2, b2, W3, b3 = unpack(params, in_dim, hidden, out_dim, bf16)
    x = np.asarray(x, dtype=np.float64)
    a1 = x @ W1 + b1
    h1 = gelu(a1)
    a2 = h1 @ W2 + b2
    h2 = gelu(a2)
    return h2 @ W3 + b3


def loss_and_grad(params, dims, x, t, bf16=True):
    """Mean squared error of forward(x) against targets t and its gradient
    with respect to the flat parameters (the gradient flows through the
    rounded weights as through the exact ones: d round(w) / dw = 1)."""
    in_dim, hidden, out_dim = dims
    W1, b1, W2, b2, W3, b3 = unpack(params, in_dim, hidden, out_dim, bf16)
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    a1 = x @ W1 + b1
    h1 = gelu(a1)
    a2 = h1 @ W2 + b2
    h2 = gelu(a2)
    y = h2 @ W3 + b3
    n = y.size
    d = y - t
    loss = float(np.sum(d * d) / n)
    dy = 2.0 * d / n
    gW3 = h2.T @ dy
    gb3 = dy.sum(axis=0)
    dh2 = dy @ W3.T
    da2 = dh2 * gelu_grad(a2)
    gW2 = h1.T @ da2
    gb2 = da2.sum(axis=0)
    dh1 = da2 @ W2.T
    da1 = dh1 * gelu_grad(a1)
    gW1 = x.T @ da1
    gb1 = da1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g
