"""Writes the oracle's per-sweep errors for the full-size parity tests.

Calls only ``oracle`` (the complex128 CPU oracle, threaded variant, which is
bit-identical to the serial one) and ``synth`` (the seeded inputs).  For each
workload below it computes the low-rank start (Alg. 1 with L = 0, rank r,
10 sweeps, then the exact embedding), runs ALS sweeps (Alg. 1) and records,
after every sweep, the training error and test error of Eq.
(BF_convergence) and the regularized objective.

    python tests/golden/make_oracle_sweeps.py [cfg3|rule16k|rule16k_ridge|all] [threads]

Workloads:
  cfg3     n = 65536, L = 12, b = 16, r = 8, omega = pi n / 16, h = 1.5,
           |Omega| = 4 n log2 n, lambda = 1e-7 (synth.config(3)), 8 sweeps
  rule16k  the same operator family at n = 16384 (L = 10) with the paper's
           sampling rule |Omega| = 6 r n log2 n (Sec. 5.1), 10 sweeps
  rule16k_ridge  rule16k with every system solved under the ridge floor
           max(lambda, 2^-20 tr(K) / dim) (the precision form's reading)
"""
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402


def rule16k_problem():
    n, L, b, r = 16384, 10, 16, 8
    return synth.make_problem("n16384_paper_rule", n, L, b, r, math.pi * n / 16, 1.5,
                              6 * r * n * int(round(math.log2(n))), 1e-7, 10, synth.SEED_BASE + 16 * 3)


RULE16K = ("n=16384 L=10 b=16 r=8 omega=pi*n/16 h=1.5 |Omega|=48 n log2 n (6 r n log2 n, Sec. 5.1) "
           "lambda=1e-7 seed=synth.SEED_BASE+48")

# name: (problem, sweeps, description, ridge floor of every system's solve)
WORKLOADS = {
    "cfg3": (lambda: synth.config(3), 8,
             "n=65536 L=12 b=16 r=8 omega=pi*n/16 h=1.5 |Omega|=4 n log2 n lambda=1e-7 (synth.config(3))", 0.0),
    "rule16k": (rule16k_problem, 10, RULE16K, 0.0),
    # the same sweeps under the complex64 precision form's reading of the
    # regularization: every system solved with max(lambda, 2^-20 tr(K) / dim)
    "rule16k_ridge": (rule16k_problem, 10, RULE16K + " ridge_rel=2^-20", 2.0 ** -20),
}


def oracle_start(p):
    """Low-rank start of the oracle: Alg. 1 with L = 0 (rank r, 10 sweeps)
    from synth.random_lowrank_start, embedded exactly into the butterfly."""
    A0, B0 = synth.random_lowrank_start(p, p.r)
    A, B = oracle.lr_complete(p.n, p.r, p.lam, A0, B0, p.i, p.j, p.t, 10)
    return oracle.embed_lowrank(p.n, p.L, p.b, p.r, A, B)


def run(name, threads):
    make, sweeps, desc, ridge = WORKLOADS[name]
    p = make()
    out = os.path.join(HERE, f"oracle_sweeps_{name}.txt")
    with oracle.threads(threads):
        t0 = time.time()
        X = oracle_start(p)
        rows = [(0, oracle.rel_err(p.n, p.L, p.b, p.r, X, p.i, p.j, p.t),
                 oracle.rel_err(p.n, p.L, p.b, p.r, X, p.it, p.jt, p.tt),
                 oracle.objective(p.n, p.L, p.b, p.r, p.lam, X, p.i, p.j, p.t))]
        print(f"{name}: start {rows[-1]} ({time.time() - t0:.0f} s)", flush=True)
        for s in range(1, sweeps + 1):
            X, st = oracle.als_sweep(p.n, p.L, p.b, p.r, p.lam, X, p.i, p.j, p.t, ridge_rel=ridge)
            te = oracle.rel_err(p.n, p.L, p.b, p.r, X, p.it, p.jt, p.tt)
            rows.append((s, st["train_rel_err"], te, st["objective"]))
            print(f"{name}: sweep {s} {rows[-1]} ({time.time() - t0:.0f} s)", flush=True)
    with open(out, "w") as f:
        f.write(f"# Oracle (complex128, Alg. 1) per-sweep errors: {desc}\n")
        f.write("# start: low-rank completion (Alg. 1 with L = 0, R = r, 10 sweeps) from\n")
        f.write("# synth.random_lowrank_start, embedded exactly (z1 = A, slices = I, zL = B)\n")
        f.write("# written by tests/golden/make_oracle_sweeps.py (oracle and synth only)\n")
        f.write(f"# nnz_train={p.nnz} ntest={p.it.size}\n")
        f.write("# sweep train_rel_err test_rel_err objective\n")
        for s, tr, te, ob in rows:
            f.write(f"{s} {tr:.17e} {te:.17e} {ob:.17e}\n")
    print(f"wrote {out}")


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "all"
    threads = int(sys.argv[2]) if len(sys.argv) > 2 else oracle.max_threads()
    for name in (WORKLOADS if which == "all" else [which]):
        run(name, threads)
