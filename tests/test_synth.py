"""Checks of the seeded input generators shared by the oracle and the CUDA path."""
import cmath
import math

import numpy as np

import synth


def test_splitmix64_published_sequence():
    # First outputs of the reference splitmix64.c for seed 1234567.
    assert [int(v) for v in synth.SplitMix64(1234567).next_u64(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_stream_is_counter_based():
    a = synth.SplitMix64(42)
    first = a.next_u64(10)
    b = synth.SplitMix64(42)
    parts = np.concatenate([b.next_u64(3), b.next_u64(7)])
    np.testing.assert_array_equal(first, parts)


def test_uniform_and_normal_moments():
    rng = synth.SplitMix64(5)
    u = rng.uniform(200000)
    assert u.min() > 0 and u.max() <= 1
    assert abs(u.mean() - 0.5) < 5e-3
    z = synth.SplitMix64(6).normal(200000)
    assert abs(z.mean()) < 1e-2 and abs(z.var() - 1) < 2e-2
    c = synth.SplitMix64(7).cnormal(100000, 2.0)
    assert abs(np.mean(np.abs(c) ** 2) - 4.0) < 0.1


def test_below_is_in_range_and_uniform():
    x = synth.SplitMix64(9).below(7, 70000)
    counts = np.bincount(x.astype(np.int64), minlength=7)
    assert counts.min() > 9500 and counts.max() < 10500


def test_draw_pairs_distinct_in_range():
    for n, cnt in [(16, 256), (64, 3000), (4096, 100000)]:
        i, j = synth.draw_pairs(n, cnt, 123)
        assert i.dtype == np.int32 and j.dtype == np.int32
        assert i.min() >= 0 and i.max() < n and j.min() >= 0 and j.max() < n
        q = i.astype(np.int64) * n + j
        assert np.unique(q).size == cnt


def test_helmholtz_kernel_closed_form():
    n, omega, h = 64, 25.0, 1.5
    for (i, j) in [(0, 0), (3, 60), (63, 1)]:
        rho = math.hypot((i + 0.5) / n - (j + 0.5) / n, h)
        want = cmath.exp(1j * omega * rho) / rho
        got = synth.helmholtz_line(n, omega, h, np.array([i]), np.array([j]))[0]
        assert abs(got - want) < 1e-15 * abs(want)


def test_config_sizes_and_split():
    p = synth.config(1)
    assert (p.n, p.L, p.b, p.r) == (256, 4, 16, 4)
    assert p.nnz + p.it.size == 8 * 256 * 8
    assert p.it.size == int(0.1 * 8 * 256 * 8)
    p2 = synth.config(2, n_override=512)
    assert (p2.n, p2.L, p2.r) == (512, 5, 6)
    # noise is 1e-4 relative
    rel = np.linalg.norm(p2.t - p2.t_clean) / np.linalg.norm(p2.t_clean)
    assert 5e-5 < rel < 2e-4


def test_batch_problem_ranges():
    probs = synth.batch_problems(8, n_choices=(256, 512))
    for p in probs:
        assert p.n in (256, 512) and p.r in (4, 6, 8)
        assert math.pi * p.n / 16 <= p.omega <= math.pi * p.n / 4
        assert 0.5 <= p.h <= 2.0


def test_family_member_equals_a_fresh_problem_at_the_same_positions():
    """A family member (same seed, other omega and h) built from a base
    problem's positions equals the problem drawn from scratch."""
    n, L, b, r = 256, 4, 16, 4
    base = synth.make_problem("a", n, L, b, r, 0.1 * math.pi * n, 1.0, 8 * n * 8, 1e-7, 15, 123)
    ref = synth.make_problem("b", n, L, b, r, 0.2 * math.pi * n, 1.5, 8 * n * 8, 1e-7, 15, 123)
    m = synth.family_member(base, "b", 0.2 * math.pi * n, 1.5)
    for f in ("i", "j", "t", "it", "jt", "tt"):
        np.testing.assert_array_equal(getattr(m, f), getattr(ref, f))
    assert (m.omega, m.h) == (ref.omega, ref.h)
