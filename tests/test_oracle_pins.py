"""Pins of the complex128 oracle against facts fixed by the paper and by
mathematics, each independent of the oracle's own code:

* the decode example printed in Fig. 2 and plain binary expansion (Eq. indices);
* a brute-force einsum contraction of the whole tensor network (Eq.
  BF_tensor_rep), with the factor tensors taken from the packed vector by
  numpy reshapes of the App. A.2 layout;
* the complementary low-rank property of Sec. 2.1 on the dense matrix;
* gauge invariance on every bond (a wrong bit assignment breaks it);
* every block of an ALS sweep equals the LAPACK least-squares solution of
  its own regularized problem (Alg. 1 solves these exactly);
* monotone regularized objective, exact low-rank recovery at L = 0, planted
  butterfly recovery, central finite differences for the gradient, and the
  vanishing gradient of the block that was minimized last.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


from helpers import envs_numpy, join_packed, lstsq_block, split_packed  # noqa: E402


def dense_by_einsum(packed, n, L, b, r):
    """Whole-matrix contraction of Eq. (BF_tensor_rep) with numpy.einsum.
    Axis order of each reshaped factor follows the MSB-first psi^{-1} of
    App. A.2: Z[m] -> (i_0..i_{L-m}, j_0..j_{m-1}, r_m, r_{m+1})."""
    z1, Z, zL = split_packed(packed, n, L, b, r)
    letters = iter("abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ")
    ib = [next(letters) for _ in range(L + 1)]       # i_0 .. i_L
    jb = [next(letters) for _ in range(L + 1)]       # j_0 .. j_L
    rk = [None] + [next(letters) for _ in range(L + 1)]  # r_1 .. r_{L+1}
    ops, subs = [], []
    ops.append(z1.reshape((2,) * L + (b, r)))
    subs.append("".join(ib) + rk[1])
    for m in range(1, L + 1):
        ops.append(Z[m - 1].reshape((2,) * (L + 1) + (r, r)))
        subs.append("".join(ib[: L - m + 1]) + "".join(jb[:m]) + rk[m] + rk[m + 1])
    ops.append(zL.reshape((2,) * L + (b, r)))
    subs.append("".join(jb) + rk[L + 1])
    expr = ",".join(subs) + "->" + "".join(ib) + "".join(jb)
    X = np.einsum(expr, *ops, optimize="greedy")
    return X.reshape(n, n)


def small_problem(n, L, b, r, seed, n_obs=None, lam=1e-9, sigma=None):
    packed = synth.random_factors(n, L, r, seed, sigma)
    if n_obs is None:
        n_obs = min(n * n, 8 * n * max(1, int(math.log2(n))))
    i, j = synth.draw_pairs(n, n_obs, seed + 1)
    return packed, i, j


# ---------------------------------------------------------------- decode

def test_fig2_decode_golden():
    with open(os.path.join(GOLDEN, "fig2_decode.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert rows == [["2", "2c+a", "c+b", "1,0,a", "0,1,b"]]
    for c in (1, 2, 3, 4, 16):
        for a in range(c):
            for bb in range(c):
                assert oracle.tree_bits(2 * c + a, 2, c) == [1, 0, a]
                assert oracle.tree_bits(c + bb, 2, c) == [0, 1, bb]


@pytest.mark.parametrize("L,b", [(0, 8), (1, 3), (4, 4), (8, 16), (5, 5)])
def test_tree_bits_are_binary_expansion(L, b):
    n = b << L
    for i in range(n):
        expect = [int(ch) for ch in format(i // b, f"0{L}b")] if L else []
        assert oracle.tree_bits(i, L, b) == expect + [i % b]


def test_slice_id_matches_prefix_formula_exhaustive():
    # slice id = (top L-m+1 bits of i//b) followed by (top m bits of j//b)
    for (L, b) in [(3, 2), (4, 3), (5, 1)]:
        n = b << L
        for m in range(1, L + 1):
            for i in range(n):
                for j in range(n):
                    pi, pj = i // b, j // b
                    k = ((pi >> (m - 1)) << m) | (pj >> (L - m))
                    assert oracle.slice_id(i, j, m, L, b) == k


def test_psi_inv_msb_first():
    assert oracle.psi_inv([1, 0, 1, 1]) == 11
    assert oracle.psi_inv([0, 0, 0, 1]) == 1
    assert oracle.psi_inv([1]) == 1


def test_num_params_closed_form_and_block_count():
    # 2nr + L 2^{L+1} r^2 (App. A.2 reshape) equals the block count of the
    # block-sparse factors of Sec. 2.2: 2^L outer c x r blocks per side and,
    # per inner level, 2^L transfer blocks of size 2r x r.
    for (n, L, b, r, expect) in [(256, 4, 16, 4, 4096), (4096, 8, 16, 6, 196608),
                                 (65536, 12, 16, 8, 7340032)]:
        blocks = 2 * ((1 << L) * b * r) + L * ((1 << L) * 2 * r * r)
        assert oracle.num_params(n, L, b, r) == expect == blocks


def test_paper_printed_counts():
    with open(os.path.join(GOLDEN, "paper_counts.txt")) as f:
        rows = [ln.split()[:3] for ln in f if ln.strip() and not ln.startswith("#")]
    for n, fac, count in rows:
        assert int(fac) * int(n) * int(round(math.log2(int(n)))) == int(count)


# ------------------------------------------------------------------ eval

@pytest.mark.parametrize("L,b,r", [(0, 5, 2), (1, 2, 2), (2, 3, 2), (3, 2, 3), (4, 2, 2)])
def test_eval_matches_dense_einsum(L, b, r):
    n = b << L
    packed = synth.random_factors(n, L, r, 7 + L)
    X = dense_by_einsum(packed, n, L, b, r)
    i, j = synth.random_pairs_full(n)
    x = oracle.eval_entries(n, L, b, r, packed, i, j)
    np.testing.assert_allclose(x, X.ravel(), rtol=0, atol=1e-13 * np.abs(X).max())


def test_eval_matches_explicit_rank_sum():
    # Literal sum over all rank tuples (r_1..r_{L+1}) for a few entries.
    n, L, b, r = 16, 2, 4, 2
    packed = synth.random_factors(n, L, r, 99)
    z1, Z, zL = split_packed(packed, n, L, b, r)
    Zt = [Z[m].reshape((2,) * (L + 1) + (r, r)) for m in range(L)]
    for (i, j) in [(0, 0), (5, 11), (15, 2), (9, 9)]:
        ib = oracle.tree_bits(i, L, b)
        jb = oracle.tree_bits(j, L, b)
        total = 0j
        for rs in itertools.product(range(r), repeat=L + 1):
            term = z1[i, rs[0]]
            for m in range(1, L + 1):
                idx = tuple(ib[: L - m + 1]) + tuple(jb[:m]) + (rs[m - 1], rs[m])
                term *= Zt[m - 1][idx]
            term *= zL[j, rs[L]]
            total += term
        x = oracle.eval_entries(n, L, b, r, packed, [i], [j])[0]
        assert abs(x - total) < 1e-13 * max(1.0, abs(total))


def test_complementary_low_rank_property():
    # Sec. 2.1: every block T(tau^l_i, nu^{L-l}_j) has rank <= r.
    n, L, b, r = 64, 4, 4, 2
    packed = synth.random_factors(n, L, r, 5)
    i, j = synth.random_pairs_full(n)
    X = oracle.eval_entries(n, L, b, r, packed, i, j).reshape(n, n)
    for l in range(L + 1):
        rows = n >> l
        cols = n >> (L - l)
        for bi in range(1 << l):
            for bj in range(1 << (L - l)):
                blk = X[bi * rows:(bi + 1) * rows, bj * cols:(bj + 1) * cols]
                sv = np.linalg.svd(blk, compute_uv=False)
                if min(blk.shape) > r:
                    assert sv[r] < 1e-10 * sv[0]
    # and the matrix as a whole is not low rank (so the check has teeth)
    sv = np.linalg.svd(X, compute_uv=False)
    assert sv[4 * r] > 1e-3 * sv[0]


def test_gauge_invariance_every_bond():
    n, L, b, r = 32, 3, 4, 3
    packed = synth.random_factors(n, L, r, 11)
    i, j = synth.random_pairs_full(n)
    x0 = oracle.eval_entries(n, L, b, r, packed, i, j)
    rng = np.random.default_rng(3)
    for bond in range(L + 1):          # bond between factor S^{bond+1} and S^{bond+2}
        z1, Z, zL = (a.copy() for a in split_packed(packed, n, L, b, r))
        G = rng.standard_normal((1 << L, r, r)) + 1j * rng.standard_normal((1 << L, r, r))
        G += 3 * np.eye(r)
        Gi = np.linalg.inv(G)
        # left factor of the bond: shared bits are all of its index bits
        # except i_{L-bond} (bit position `bond` of its slice id)
        if bond == 0:
            for i_ in range(n):
                z1[i_] = z1[i_] @ G[i_ // b]
        else:
            for k in range(1 << (L + 1)):
                g = ((k >> (bond + 1)) << bond) | (k & ((1 << bond) - 1))
                Z[bond - 1, k] = Z[bond - 1, k] @ G[g]
        # right factor of the bond: shared bits drop j_bond (bit 0)
        if bond == L:
            for j_ in range(n):
                zL[j_] = Gi[j_ // b] @ zL[j_]
        else:
            for k in range(1 << (L + 1)):
                Z[bond, k] = Gi[k >> 1] @ Z[bond, k]
        x1 = oracle.eval_entries(n, L, b, r, join_packed(z1, Z, zL), i, j)
        np.testing.assert_allclose(x1, x0, rtol=0, atol=1e-11 * np.abs(x0).max())


# ------------------------------------------------------------------- ALS

def test_every_als_block_is_the_exact_regularized_lstsq():
    n, L, b, r = 64, 3, 8, 2
    lam = 1e-3
    packed, i, j = small_problem(n, L, b, r, seed=21, n_obs=1500)
    t = synth.helmholtz_line(n, math.pi * n / 8, 1.0, i, j)
    new, _ = oracle.als_sweep(n, L, b, r, lam, packed, i, j, t)
    z1o, Zo, zLo = split_packed(packed, n, L, b, r)
    z1n, Zn, zLn = split_packed(new, n, L, b, r)
    pi, pj = i // b, j // b

    def check(got, want):
        scale = max(np.abs(want).max(), 1e-30)
        assert np.abs(got - want).max() < 1e-9 * scale

    # S^1: design = full right env from the old factors
    _, w_old = envs_numpy(z1o, Zo, zLo, i, j, L, b, r)
    for row in range(n):
        sel = np.nonzero(i == row)[0]
        check(z1n[row], lstsq_block(w_old[0][sel], t[sel], lam))
    # middle factors: left env from new factors, right env from old ones
    for m in range(1, L + 1):
        Zmix = np.concatenate([Zn[: m - 1], Zo[m - 1:]])
        h_new, _ = envs_numpy(z1n, Zmix, zLo, i, j, L, b, r)
        _, w_o = envs_numpy(z1o, Zo, zLo, i, j, L, b, r)
        key = ((pi >> (m - 1)) << m) | (pj >> (L - m))
        for k in range(1 << (L + 1)):
            sel = np.nonzero(key == k)[0]
            A = np.einsum("ea,ec->eac", h_new[m][sel], w_o[m][sel]).reshape(len(sel), r * r)
            check(Zn[m - 1, k].ravel(), lstsq_block(A, t[sel], lam))
    # S^{L+2}: design = full left env from the new factors
    h_new, _ = envs_numpy(z1n, Zn, zLo, i, j, L, b, r)
    for col in range(n):
        sel = np.nonzero(j == col)[0]
        check(zLn[col], lstsq_block(h_new[L + 1][sel], t[sel], lam))


def test_regularized_objective_monotone():
    p = synth.config(1)
    A, B = synth.random_lowrank_start(p, p.r)
    A, B = oracle.lr_complete(p.n, p.r, p.lam, A, B, p.i, p.j, p.t, 10)
    X = oracle.embed_lowrank(p.n, p.L, p.b, p.r, A, B)
    f_prev = oracle.objective(p.n, p.L, p.b, p.r, p.lam, X, p.i, p.j, p.t)
    for _ in range(6):
        X, st = oracle.als_sweep(p.n, p.L, p.b, p.r, p.lam, X, p.i, p.j, p.t)
        assert st["objective"] <= f_prev * (1 + 1e-12)
        f_prev = st["objective"]


def test_lowrank_special_case_recovers_full_observation():
    # L = 0: Alg. 1 is ALS matrix completion (Sec. 4.1.1 remark).  With all
    # entries observed and lambda = 0 one sweep recovers a rank-R matrix.
    n, R = 24, 3
    rng = synth.SplitMix64(77)
    As = rng.cnormal(n * R).reshape(n, R)
    Bs = rng.cnormal(n * R).reshape(n, R)
    T = As @ Bs.T
    i, j = synth.random_pairs_full(n)
    A0 = rng.cnormal(n * R).reshape(n, R)
    B0 = rng.cnormal(n * R).reshape(n, R)
    A, B = oracle.lr_complete(n, R, 0.0, A0, B0, i, j, T.ravel(), 2)
    assert np.abs(A @ B.T - T).max() < 1e-12 * np.abs(T).max()


def test_planted_butterfly_recovery():
    n, L, b, r = 256, 4, 16, 3
    planted = synth.random_factors(n, L, r, 1234)
    i, j = synth.draw_pairs(n, 8 * n * 8, 4321)
    t = oracle.eval_entries(n, L, b, r, planted, i, j)
    ntest = len(i) // 10
    it, jt, tt = i[-ntest:], j[-ntest:], t[-ntest:]
    i, j, t = i[:-ntest], j[:-ntest], t[:-ntest]
    noise = synth.SplitMix64(99).cnormal(planted.size, 1e-2)
    X = planted * (1 + noise)
    errs = []
    for _ in range(40):
        X, _ = oracle.als_sweep(n, L, b, r, 1e-12, X, i, j, t)
        errs.append(oracle.rel_err(n, L, b, r, X, it, jt, tt))
    # linear convergence to the planted operator (held-out entries)
    assert errs[-1] < 1e-11
    assert all(b_ < a_ for a_, b_ in zip(errs[:-1], errs[1:]))


def test_singular_block_kept_and_counted():
    # lambda = 0 and an empty row: that fiber's system is singular.
    n, L, b, r = 16, 1, 8, 2
    packed = synth.random_factors(n, L, r, 3)
    i, j = synth.draw_pairs(n, 200, 5)
    keep = i != 3
    i, j = i[keep], j[keep]
    t = synth.helmholtz_line(n, 10.0, 1.0, i, j)
    new, st = oracle.als_sweep(n, L, b, r, 0.0, packed, i, j, t)
    assert st["singular"] >= 1
    np.testing.assert_array_equal(new[3 * r:4 * r], packed[3 * r:4 * r])


def test_empty_slice_with_lambda_becomes_zero():
    n, L, b, r = 16, 1, 8, 2
    packed = synth.random_factors(n, L, r, 3)
    i, j = synth.draw_pairs(n, 200, 5)
    keep = i != 3
    i, j = i[keep], j[keep]
    t = synth.helmholtz_line(n, 10.0, 1.0, i, j)
    new, st = oracle.als_sweep(n, L, b, r, 1e-3, packed, i, j, t)
    assert st["singular"] == 0
    assert np.all(new[3 * r:4 * r] == 0)


# -------------------------------------------------------------- gradient

def test_gradient_central_differences():
    n, L, b, r = 32, 2, 8, 2
    lam = 1e-2
    packed, i, j = small_problem(n, L, b, r, seed=8, n_obs=300)
    t = synth.helmholtz_line(n, 20.0, 1.0, i, j)
    g, f0 = oracle.grad(n, L, b, r, lam, packed, i, j, t, include_reg=True)
    assert abs(f0 - oracle.objective(n, L, b, r, lam, packed, i, j, t)) < 1e-12 * abs(f0)
    rng = np.random.default_rng(0)
    for p in rng.choice(packed.size, 25, replace=False):
        for unit in (1.0, 1j):
            hstep = 1e-6 * max(1.0, abs(packed[p]))
            xp, xm = packed.copy(), packed.copy()
            xp[p] += unit * hstep
            xm[p] -= unit * hstep
            fd = (oracle.objective(n, L, b, r, lam, xp, i, j, t)
                  - oracle.objective(n, L, b, r, lam, xm, i, j, t)) / (2 * hstep)
            an = g[p].real if unit == 1.0 else g[p].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, np.abs(g).max())


def test_gradient_of_last_minimized_block_vanishes():
    n, L, b, r = 64, 3, 8, 2
    lam = 1e-4
    packed, i, j = small_problem(n, L, b, r, seed=31, n_obs=1200)
    t = synth.helmholtz_line(n, 30.0, 1.0, i, j)
    new, _ = oracle.als_sweep(n, L, b, r, lam, packed, i, j, t)
    g, _ = oracle.grad(n, L, b, r, lam, new, i, j, t, include_reg=True)
    _, _, gL = split_packed(g, n, L, b, r)
    g1, _, _ = split_packed(oracle.grad(n, L, b, r, lam, packed, i, j, t)[0], n, L, b, r)
    assert np.abs(gL).max() < 1e-10 * max(1.0, np.abs(g1).max())


# ------------------------------------------------------------ init / data

def test_lowrank_embedding_reproduces_product():
    n, L, b, r = 64, 3, 8, 3
    rng = synth.SplitMix64(4)
    A = rng.cnormal(n * r).reshape(n, r)
    B = rng.cnormal(n * r).reshape(n, r)
    X = oracle.embed_lowrank(n, L, b, r, A, B)
    i, j = synth.random_pairs_full(n)
    x = oracle.eval_entries(n, L, b, r, X, i, j).reshape(n, n)
    np.testing.assert_allclose(x, A @ B.T, rtol=0, atol=1e-14 * np.abs(A @ B.T).max())


def test_lowrank_start_quality_matches_paper_remark():
    # Sec. 4.2: low-rank completion with R = r leaves relative error above 0.5,
    # and an error near 0.9 is a good enough start.
    p = synth.config(1)
    A, B = synth.random_lowrank_start(p, p.r)
    A, B = oracle.lr_complete(p.n, p.r, p.lam, A, B, p.i, p.j, p.t, 10)
    X = oracle.embed_lowrank(p.n, p.L, p.b, p.r, A, B)
    tr = oracle.rel_err(p.n, p.L, p.b, p.r, X, p.i, p.j, p.t)
    te = oracle.rel_err(p.n, p.L, p.b, p.r, X, p.it, p.jt, p.tt)
    assert 0.5 < tr < 1.0 and 0.5 < te < 1.2


def test_lbfgs_monotone_and_reaches_stationarity():
    # Armijo line search: the objective never increases; a correct two-loop
    # direction drives the gradient norm down by orders of magnitude.
    n, L, b, r = 32, 2, 8, 2
    lam = 1e-3
    packed, i, j = small_problem(n, L, b, r, seed=12, n_obs=400)
    t = synth.helmholtz_line(n, 15.0, 1.0, i, j)
    g0, f0 = oracle.grad(n, L, b, r, lam, packed, i, j, t)
    X, hist = oracle.lbfgs(n, L, b, r, lam, packed, i, j, t, 120)
    assert hist[0] < f0
    assert all(b_ <= a_ * (1 + 1e-12) for a_, b_ in zip(hist[:-1], hist[1:]))
    g, f = oracle.grad(n, L, b, r, lam, X, i, j, t)
    assert abs(f - hist[-1]) <= 1e-12 * abs(f)
    assert np.linalg.norm(g) < 1e-3 * np.linalg.norm(g0)


def test_threaded_oracle_is_bit_identical_to_serial():
    """The threaded variant runs independent systems and entries on several
    threads with every sum in its serial order: sweeps, evaluations and
    errors must be identical bit for bit to the serial oracle."""
    p = synth.config(2, n_override=512)
    X0 = synth.random_factors(p.n, p.L, p.r, 17, sigma=0.4)
    out = {}
    for nt in (1, 4):
        with oracle.threads(nt):
            X1, st = oracle.als_sweep(p.n, p.L, p.b, p.r, p.lam, X0, p.i, p.j, p.t)
            X2, st2 = oracle.als_sweep(p.n, p.L, p.b, p.r, p.lam, X1, p.i, p.j, p.t)
            x = oracle.eval_entries(p.n, p.L, p.b, p.r, X2, p.it, p.jt)
            te = oracle.rel_err(p.n, p.L, p.b, p.r, X2, p.it, p.jt, p.tt)
            out[nt] = (X2, st2, x, te)
    (a, sa, xa, ta), (b_, sb, xb, tb) = out[1], out[4]
    assert np.array_equal(a.view(np.float64), b_.view(np.float64))
    assert np.array_equal(xa.view(np.float64), xb.view(np.float64))
    assert sa == sb and ta == tb


def _bfgs_matrix_direction(pairs, g):
    """-H g with H the explicit BFGS inverse-Hessian recursion over the stored
    pairs, oldest to newest: H <- (I - rho s y^T)^T-form update
    H <- V^T H V + rho s s^T with V = I - rho y s^T, from H = gamma I with
    gamma = s^T y / y^T y of the newest pair (Nocedal and Wright, eq. 7.19
    and 7.20); gamma = 1 and H = I without pairs."""
    dim = g.size
    if not pairs:
        return -g
    s_new, y_new = pairs[-1]
    H = (float(s_new @ y_new) / float(y_new @ y_new)) * np.eye(dim)
    for s_, y_ in pairs:
        rho = 1.0 / float(y_ @ s_)
        V = np.eye(dim) - rho * np.outer(y_, s_)
        H = V.T @ H @ V + rho * np.outer(s_, s_)
    return -H @ g


@pytest.mark.parametrize("n,L,b,r,memory", [(2, 1, 1, 1, 10), (2, 1, 1, 1, 3), (3, 0, 3, 1, 10),
                                            (3, 0, 3, 1, 2)])
def test_lbfgs_direction_is_the_explicit_bfgs_matrix_product(n, L, b, r, memory):
    """The two-loop recursion of oracle.lbfgs must give exactly the direction
    -H_k g_k of the explicit inverse-Hessian recursion over the last `memory`
    accepted pairs (both with full memory and truncated memory).  A wrong
    gamma pair, a swapped loop order or a dropped rho fails this check; the
    step lengths must satisfy the Armijo rule from the stated first trial."""
    lam = 1e-2
    X0 = synth.random_factors(n, L, r, 5 + n + memory, sigma=0.7)
    i, j = synth.random_pairs_full(n)
    t = synth.helmholtz_line(n, 7.0, 1.0, i, j)
    trace = []
    iters = 12
    oracle.lbfgs(n, L, b, r, lam, X0, i, j, t, iters, memory=memory, trace=trace)
    assert len(trace) == iters
    pairs = []
    for k, (x, g, d, step, f) in enumerate(trace):
        want = _bfgs_matrix_direction(pairs[-memory:], g)
        if not float(g @ want) < 0.0:
            want = -g
        np.testing.assert_allclose(d, want, rtol=1e-9, atol=1e-12 * np.abs(want).max())
        if k + 1 < len(trace):
            x1, g1, _, _, f1 = trace[k + 1]
            assert np.allclose(x1, x + step * d, rtol=0, atol=1e-14 * max(1.0, np.abs(x).max()))
            assert f1 <= f + 1e-4 * step * float(g @ d)          # Armijo, c1 = 1e-4
            s_, y_ = x1 - x, g1 - g
            if float(s_ @ y_) > 1e-12 * np.linalg.norm(s_) * np.linalg.norm(y_):
                pairs.append((s_, y_))
        if k == 0:
            first = 1.0 / np.linalg.norm(g)
            # the first trial step is 1 / ||g||, halved until Armijo holds
            assert any(abs(step - first * 0.5 ** h) <= 1e-15 * first for h in range(31))
    assert len(pairs) > memory or memory >= iters


# ----------------------------------------------------------- MLP oracle

def test_bf16_rounding_is_nearest_even():
    from oracle import mlp
    u = 2.0 ** -7   # bfloat16 spacing on [1, 2)
    vals = [1.0, 3.0, 1 + u / 2, 1 + 3 * u / 2, 1 + u / 2 + 2.0 ** -20, -(1 + 3 * u / 2), 0.0]
    want = [1.0, 3.0, 1.0, 1 + 2 * u, 1 + u, -(1 + 2 * u), 0.0]
    np.testing.assert_array_equal(mlp.bf16_round(np.array(vals)), np.array(want))


def test_gelu_closed_forms():
    from oracle import mlp
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    assert abs(mlp.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    assert abs(mlp.gelu(np.array([-10.0]))[0]) < 1e-12
    a = np.linspace(-4, 4, 17)
    hstep = 1e-6
    fd = (mlp.gelu(a + hstep) - mlp.gelu(a - hstep)) / (2 * hstep)
    np.testing.assert_allclose(mlp.gelu_grad(a), fd, rtol=1e-7, atol=1e-9)


def test_mlp_backprop_matches_finite_differences():
    from oracle import mlp
    dims = (2, 5, 7)
    _, npar = mlp.layout(*dims)
    rng = np.random.default_rng(3)
    p = rng.normal(size=npar) * 0.5
    x = rng.uniform(-1, 1, size=(4, 2))
    t = rng.normal(size=(4, 7))
    loss, g = mlp.loss_and_grad(p, dims, x, t, bf16=False)
    assert abs(loss - np.mean((mlp.forward(p, dims, x, bf16=False) - t) ** 2)) < 1e-14
    fd = np.zeros(npar)
    hstep = 1e-6
    for q in range(npar):
        e = np.zeros(npar)
        e[q] = hstep
        fd[q] = (mlp.loss_and_grad(p + e, dims, x, t, bf16=False)[0]
                 - mlp.loss_and_grad(p - e, dims, x, t, bf16=False)[0]) / (2 * hstep)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


# ----------------------------------------------------------- gauge oracle

def _random_factors(n, L, r, seed):
    rng = np.random.default_rng(seed)
    P = oracle.num_params(n, L, n >> L, r)
    return rng.normal(size=P) + 1j * rng.normal(size=P)


@pytest.mark.parametrize("n,L,b,r", [(64, 3, 8, 3), (96, 4, 6, 2), (40, 0, 40, 4)])
def test_canonical_gauge_keeps_entries_and_is_orthonormal_and_unique(n, L, b, r):
    from oracle import gauge
    X = _random_factors(n, L, r, 7)
    C = gauge.canonicalize(n, L, b, r, X)
    rng = np.random.default_rng(8)
    i = rng.integers(0, n, 300).astype(np.int32)
    j = rng.integers(0, n, 300).astype(np.int32)
    xa = oracle.eval_entries(n, L, b, r, X, i, j)
    xc = oracle.eval_entries(n, L, b, r, C, i, j)
    assert np.max(np.abs(xa - xc)) <= 1e-11 * np.max(np.abs(xa))
    # left-orthonormal: each leaf block of z1 and each stacked slice pair
    z1 = C[:n * r].reshape(n, r)
    if L > 0:
        for p in range(n // b):
            blk = z1[p * b:(p + 1) * b]
            np.testing.assert_allclose(blk.conj().T @ blk, np.eye(r), atol=1e-12)
        S = 1 << (L + 1)
        Z = C[n * r:n * r + L * S * r * r].reshape(L, S, r, r)
        for m in range(1, L + 1):
            for A in range(1 << (L - m)):
                for B in range(1 << m):
                    M = np.vstack([Z[m - 1, ((A << 1) << m) | B], Z[m - 1, ((A << 1 | 1) << m) | B]])
                    np.testing.assert_allclose(M.conj().T @ M, np.eye(r), atol=1e-12)
    # a second application changes nothing (the gauge is fixed)
    C2 = gauge.canonicalize(n, L, b, r, C)
    assert np.max(np.abs(C2 - C)) <= 1e-11 * np.max(np.abs(C))
