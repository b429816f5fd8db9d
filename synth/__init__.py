"""Seeded synthetic inputs for butterfly tensor completion.

This module is shared by the oracle, the CUDA path, the tests and the
benchmark.  It holds none of the completion method's arithmetic: it only
draws random numbers, observed index sets and the values of the operator that
is to be completed.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; the finalizer constants are
Vigna's published ones), evaluated vectorised in numpy:
    state_k = seed + k * 0x9E3779B97F4A7C15           (k = 1, 2, ...)
    z = state_k; z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB;  out = z ^ (z >> 31)

Workload (a stand-in for the paper's Green's-function experiments of Sec. 5.1,
which use 3-D grids with a KD-tree ordering): the 1-D line-to-line Helmholtz
kernel K(i, j) = exp(1j * omega * rho) / rho, rho = |x_i - y_j| with
x_i = ((i + 1/2)/n, 0) and y_j = ((j + 1/2)/n, h).  Observed entries are drawn
uniformly without replacement; the last floor(0.1 |Omega|) draws are the test
set.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
MIX1 = np.uint64(0xBF58476D1CE4E5B9)
MIX2 = np.uint64(0x94D049BB133111EB)
SEED_BASE = 0xBFC00000
BATCH_SEED_BASE = 0xBFC10000
SEED_OMEGA, SEED_NOISE, SEED_INIT, SEED_PLANT, SEED_PARAMS = 0, 1, 2, 3, 4


class SplitMix64:
    """Counter-based SplitMix64 stream (output k uses state seed + k*gamma)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.k = 0

    def next_u64(self, count: int) -> np.ndarray:
        ks = np.arange(self.k + 1, self.k + 1 + count, dtype=np.uint64)
        self.k += count
        with np.errstate(over="ignore"):
            z = self.seed + ks * GAMMA
            z = (z ^ (z >> np.uint64(30))) * MIX1
            z = (z ^ (z >> np.uint64(27))) * MIX2
        return z ^ (z >> np.uint64(31))

    def uniform(self, count: int) -> np.ndarray:
        """Doubles in (0, 1]: ((x >> 11) + 1) * 2^-53."""
        x = self.next_u64(count) >> np.uint64(11)
        return (x.astype(np.float64) + 1.0) * (2.0 ** -53)

    def normal(self, count: int) -> np.ndarray:
        """Standard normals by the Box-Muller transform."""
        half = (count + 1) // 2
        u1 = self.uniform(half)
        u2 = self.uniform(half)
        rad = np.sqrt(-2.0 * np.log(u1))
        z = np.empty(2 * half)
        z[0::2] = rad * np.cos(2.0 * np.pi * u2)
        z[1::2] = rad * np.sin(2.0 * np.pi * u2)
        return z[:count]

    def cnormal(self, count: int, sigma: float = 1.0) -> np.ndarray:
        """Circular complex Gaussians CN(0, sigma^2)."""
        z = self.normal(2 * count) * (sigma / math.sqrt(2.0))
        return z[0::2] + 1j * z[1::2]

    def below(self, bound: int, count: int) -> np.ndarray:
        """Exactly uniform integers in [0, bound) by rejection."""
        out = np.empty(0, dtype=np.uint64)
        lim = (2 ** 64 // bound) * bound
        while out.size < count:
            x = self.next_u64(max(count - out.size, 16) + 16)
            if lim < 2 ** 64:
                x = x[x < np.uint64(lim)]
            out = np.concatenate([out, x % np.uint64(bound)])
        return out[:count]


def draw_pairs(n: int, count: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """`count` distinct (i, j) pairs, uniform without replacement, in draw
    order: linear index q in [0, n^2), i = q // n, j = q % n."""
    total = n * n
    if count > total:
        raise ValueError("more entries requested than the matrix has")
    rng = SplitMix64(seed)
    kept = np.empty(0, dtype=np.uint64)
    while kept.size < count:
        need = count - kept.size
        cand = rng.below(total, need + need // 4 + 64)
        allq = np.concatenate([kept, cand])
        _, first = np.unique(allq, return_index=True)
        kept = allq[np.sort(first)]
    q = kept[:count].astype(np.int64)
    return (q // n).astype(np.int32), (q % n).astype(np.int32)


def helmholtz_line(n: int, omega: float, h: float, i: np.ndarray, j: np.ndarray) -> np.ndarray:
    """K(i, j) = exp(1j omega rho) / rho on two parallel lines at distance h."""
    xi = (np.asarray(i, dtype=np.float64) + 0.5) / n
    yj = (np.asarray(j, dtype=np.float64) + 0.5) / n
    rho = np.hypot(xi - yj, h)
    return np.exp(1j * omega * rho) / rho


def radon_1d(n: int, i: np.ndarray, j: np.ndarray) -> np.ndarray:
    """The discretized 1-D Radon transform of Sec. 5.3: t = exp(2 pi 1j phi),
    phi(x, y) = x y + c(x) |y|, c(x) = (2 + sin(2 pi x)) / 8, with
    x = i' / n and y = j' - n / 2 for the 1-based indices i' = i + 1,
    j' = j + 1."""
    x = (np.asarray(i, dtype=np.float64) + 1.0) / n
    y = (np.asarray(j, dtype=np.float64) + 1.0) - n / 2.0
    c = (2.0 + np.sin(2.0 * np.pi * x)) / 8.0
    phi = x * y + c * np.abs(y)
    # the phase only matters modulo 1: reduce it before the exponential
    return np.exp(2j * np.pi * (phi - np.floor(phi)))


@dataclass
class Problem:
    """One completion problem: sizes, hyper-parameters and observed data."""
    name: str
    n: int
    L: int
    b: int
    r: int
    omega: float
    h: float
    lam: float
    sweeps: int
    seed: int
    i: np.ndarray = field(repr=False, default=None)      # training rows (int32)
    j: np.ndarray = field(repr=False, default=None)      # training cols (int32)
    t: np.ndarray = field(repr=False, default=None)      # training values (complex128)
    it: np.ndarray = field(repr=False, default=None)     # test rows
    jt: np.ndarray = field(repr=False, default=None)     # test cols
    tt: np.ndarray = field(repr=False, default=None)     # test values
    t_clean: np.ndarray = field(repr=False, default=None)  # training values before noise

    @property
    def nnz(self) -> int:
        return int(self.i.size)


def make_problem(name: str, n: int, L: int, b: int, r: int, omega: float, h: float,
                 n_obs: int, lam: float, sweeps: int, seed: int,
                 noise_rel: float = 0.0, test_frac: float = 0.1) -> Problem:
    if n != b * (1 << L):
        raise ValueError("n must equal b * 2^L")
    i, j = draw_pairs(n, n_obs, seed + SEED_OMEGA)
    vals = helmholtz_line(n, omega, h, i, j)
    clean = vals.copy()
    if noise_rel > 0.0:
        rms = math.sqrt(float(np.mean(np.abs(vals) ** 2)))
        vals = vals + SplitMix64(seed + SEED_NOISE).cnormal(vals.size, noise_rel * rms)
    n_test = int(math.floor(test_frac * n_obs))
    n_train = n_obs - n_test
    return Problem(name=name, n=n, L=L, b=b, r=r, omega=omega, h=h, lam=lam,
                   sweeps=sweeps, seed=seed,
                   i=i[:n_train].copy(), j=j[:n_train].copy(), t=vals[:n_train].copy(),
                   it=i[n_train:].copy(), jt=j[n_train:].copy(), tt=vals[n_train:].copy(),
                   t_clean=clean[:n_train].copy())


def family_member(base: Problem, name: str, omega: float, h: float) -> Problem:
    """A member of `base`'s operator family at the same sample positions
    (training and test) with the kernel's parameters (omega, h) changed:
    only the values are recomputed (noise-free)."""
    tr = helmholtz_line(base.n, omega, h, base.i, base.j)
    te = helmholtz_line(base.n, omega, h, base.it, base.jt)
    return Problem(name=name, n=base.n, L=base.L, b=base.b, r=base.r, omega=omega, h=h, lam=base.lam,
                   sweeps=base.sweeps, seed=base.seed, i=base.i, j=base.j, t=tr, it=base.it, jt=base.jt,
                   tt=te, t_clean=tr)


def config(index: int, n_override: int | None = None) -> Problem:
    """The single-problem workloads, by 1-based index:
    1  n=256   L=4  b=16 r=4 h=1   omega=pi n/8  |Omega|=8 n log2 n  lambda=1e-8 10 sweeps
    2  n=4096  L=8  b=16 r=6 h=1   omega=pi n/8  |Omega|=6 n log2 n  lambda=1e-7 20 sweeps,
       complex Gaussian noise at 1e-4 relative
    3  n=65536 L=12 b=16 r=8 h=1.5 omega=pi n/16 |Omega|=4 n log2 n  lambda=1e-7 20 sweeps
    5  n=4096  L=8  b=16 r=6 h=1   omega=pi n/8  |Omega|=6 n log2 n  lambda=1e-7 20 sweeps
    `n_override` keeps b, r, h, the omega/n ratio and the sampling factor but
    changes n (for reduced-size runs of the same workload)."""
    table = {
        1: dict(n=256, b=16, r=4, h=1.0, wfac=1 / 8, c=8, lam=1e-8, sweeps=10, noise=0.0),
        2: dict(n=4096, b=16, r=6, h=1.0, wfac=1 / 8, c=6, lam=1e-7, sweeps=20, noise=1e-4),
        3: dict(n=65536, b=16, r=8, h=1.5, wfac=1 / 16, c=4, lam=1e-7, sweeps=20, noise=0.0),
        5: dict(n=4096, b=16, r=6, h=1.0, wfac=1 / 8, c=6, lam=1e-7, sweeps=20, noise=0.0),
    }
    p = table[index]
    n = n_override or p["n"]
    L = int(round(math.log2(n // p["b"])))
    n_obs = int(p["c"] * n * int(round(math.log2(n))))
    return make_problem(f"cfg{index}" + (f"_n{n}" if n_override else ""), n, L, p["b"], p["r"],
                        math.pi * n * p["wfac"], p["h"], n_obs, p["lam"], p["sweeps"],
                        SEED_BASE + 16 * index, noise_rel=p["noise"])


RADON_SEED_BASE = 0xBFC20000


def radon_problem(n: int = 4096, b: int = 4, r: int = 12, c_obs: float = 70.0, c_test: float = 10.0,
                  lam: float = 1e-8, sweeps: int = 20) -> Problem:
    """The Radon-transform workload of Sec. 5.3: the matrix of radon_1d,
    leaf size b (the paper's c = 4), rank estimate r, |Omega| = c_obs n log2 n
    training and |Omega_test| = c_test n log2 n test entries, drawn uniformly
    without replacement (the test entries are the last draws).  The default is
    the paper's convergence study: n = 4096 (L = 10), rank estimate r = 12,
    3,440,640 training and 491,520 test entries (the printed counts, which are
    7 r n log2 n and r n log2 n with the actual rank 10)."""
    L = int(round(math.log2(n // b)))
    if n != b << L:
        raise ValueError("n must equal b * 2^L")
    n_train = int(round(c_obs * n * math.log2(n)))
    n_test = int(round(c_test * n * math.log2(n)))
    n_obs = n_train + n_test
    seed = RADON_SEED_BASE + 16 * int(round(math.log2(n)))
    i, j = draw_pairs(n, n_obs, seed + SEED_OMEGA)
    vals = radon_1d(n, i, j)
    return Problem(name=f"radon_n{n}", n=n, L=L, b=b, r=r, omega=0.0, h=0.0, lam=lam, sweeps=sweeps,
                   seed=seed, i=i[:n_train].copy(), j=j[:n_train].copy(), t=vals[:n_train].copy(),
                   it=i[n_train:].copy(), jt=j[n_train:].copy(), tt=vals[n_train:].copy(),
                   t_clean=vals[:n_train].copy())


def lr2bf_gaussians(n: int, L: int, b: int, r: int, p: int, seed: int) -> np.ndarray:
    """The Gaussian sketch matrices of the randomized low-rank to butterfly
    conversion, CN(0, 1) from SplitMix64(seed), packed in the order the
    conversion reads them: O_0 (n rows), then the left levels l = 1 .. H
    (H = floor(L / 2)) and the right levels l = 1 .. L - H, b 2^{L-l} rows
    each; r + p columns, row-major."""
    H = L // 2
    rows = n + sum(b << (L - l) for l in range(1, H + 1)) + sum(b << (L - l) for l in range(1, L - H + 1))
    return SplitMix64(seed).cnormal(rows * (r + p))


def batch_problems(count: int = 64, seed_base: int = BATCH_SEED_BASE,
                   n_choices=(1024, 2048, 4096, 8192, 16384), paper_rule: bool = False) -> list[Problem]:
    """The batched workload: independent problems with n drawn from
    `n_choices` (b = 16), r uniform in {4, 6, 8}, omega ~ U[pi n/16, pi n/4],
    receiver offset h ~ U[0.5, 2], |Omega| = c n log2 n with c ~ U[4, 8]
    (or, with paper_rule, the paper's 6 r n log2 n)."""
    out = []
    for p in range(count):
        rng = SplitMix64(seed_base + 16 * p + SEED_PARAMS)
        u = rng.uniform(5)
        n = int(n_choices[min(int(u[0] * len(n_choices)), len(n_choices) - 1)])
        r = (4, 6, 8)[min(int(u[1] * 3), 2)]
        omega = math.pi * n * (1 / 16 + u[2] * (1 / 4 - 1 / 16))
        h = 0.5 + 1.5 * u[3]
        c = 4.0 + 4.0 * u[4]
        L = int(round(math.log2(n // 16)))
        n_obs = int(round((6 * r if paper_rule else c) * n * math.log2(n)))
        out.append(make_problem(f"batch{p}", n, L, 16, r, omega, h, n_obs, 1e-7, 20,
                                seed_base + 16 * p))
    return out


def random_lowrank_start(prob: Problem, R: int) -> tuple[np.ndarray, np.ndarray]:
    """Seeded CN(0, sigma^2) starting factors A, B (n x R) for low-rank
    completion, sigma = (rms(t) / R)^(1/2) so that A B^T has the data's scale."""
    rms = math.sqrt(float(np.mean(np.abs(prob.t) ** 2)))
    sigma = math.sqrt(rms / R)
    rng = SplitMix64(prob.seed + SEED_INIT)
    A = rng.cnormal(prob.n * R, sigma).reshape(prob.n, R)
    B = rng.cnormal(prob.n * R, sigma).reshape(prob.n, R)
    return A, B


def random_factors(n: int, L: int, r: int, seed: int, sigma: float | None = None) -> np.ndarray:
    """Packed complex128 factor vector with i.i.d. CN(0, sigma^2) entries
    (default sigma^2 = 1/r), length 2 n r + L 2^{L+1} r^2."""
    P = 2 * n * r + L * (1 << (L + 1)) * r * r
    s = math.sqrt(1.0 / r) if sigma is None else sigma
    return SplitMix64(seed).cnormal(P, s)


def random_pairs_full(n: int) -> tuple[np.ndarray, np.ndarray]:
    """All n^2 index pairs in row-major order (for tiny exhaustive checks)."""
    q = np.arange(n * n, dtype=np.int64)
    return (q // n).astype(np.int32), (q % n).astype(np.int32)
