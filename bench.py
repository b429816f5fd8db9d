#!/usr/bin/env python
"""Benchmark: ALS sweep entries/s for butterfly completion on one GB300.

Workload (the n = 65536 precision-form problem): n = 65536, L = 12, b = 16,
r = 8, omega = pi n / 16, receiver line at h = 1.5, |Omega| = 4 n log2 n
(3,774,874 training / 419,430 test entries), lambda = 1e-7, complex64 chains
with compensated normal-equation sums and FP64 per-slice solves.  Inputs are
seeded synthetic data (synth.config(3)); the start is the low-rank completion
start (Sec. 4.2) computed on the GPU.

A step is one full ALS sweep (Alg. 1: right environments, S^1 fibers, the L
middle factors, S^{L+2} fibers, training / test error and objective).  The
working set (about 4.5 GB of environments, values and orders) is far larger
than L2, so no flush is needed between steps.

Lines printed (one JSON line, rank 0):
  value      entries/s of the timed sweeps (replays of the captured sweep
             graph), whole job (sum over ranks)
  e2e        the same through the public API with host buffers: every step
             copies the factors from pinned host memory, sweeps, and copies
             the factors and statistics back
  kernels_ms per-kernel CUDA-event times of the same number of sweeps run
             again with the library's profiling on
  roofline   dominant kernel (the per-slice normal-equation kernel)
  kernel_rooflines  every kernel above 1 % of a sweep against its bound
  gradient   one full gradient (bfc_grad, device-resident) and the roofline
             of its middle-level kernel
  time_to_1e-3_test_error, batched, learned_start  the three forms against
             plain FP64 ALS on the same GPU
  cpu_baseline  the complex128 oracle timed on a bounded sample (rank 0)
Multi-GPU: every rank runs an independent replica (the single problem does
not shard without an exchange step); value is the sum over ranks.

--impl reference times the oracle as it stands on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ALS sweep entries/s (n=65536 precision form)"
UNIT = "entries/s"
WORKLOAD = ("n=65536 L=12 b=16 r=8, exp(i w rho)/rho line-to-line kernel, w=pi n/16, h=1.5, "
            "|Omega|=4 n log2 n (3774874 train / 419430 test), lambda=1e-7")
TC_FLOPS_PER_ENTRY = 2 * 3 * 128 * 144   # flop, one contraction position x M 128 x N 144 x 3 products
# DRAM counters of one k_mid_gram_tc launch (ncu, n = 32768, L = 11: 1,769,472
# entries, 4096 slices), valid for the kernel source with this sha256 prefix
TC_GRAM_TRAFFIC = {"source": "paper_2510_17734_gb300/csrc/bfc_gram_tc.cuh", "sha": "8159f55fbacf40ac",
                   "read_bytes": 241.090048e6, "write_bytes": 51.348736e6, "entries": 1769472, "slices": 4096}


# DRAM counters of k_mid_solve at the n = 65536 workload itself (ncu, one-pass
# metrics, mean of two launches of the first sweep: 3,774,874 entries, 8192
# slices per level), valid for the kernel source with this sha256 prefix
SOLVE_TRAFFIC = {"source": "paper_2510_17734_gb300/csrc/bfc_kernels.cuh", "sha": "fca9bdd68955b392",
                 # the kernel and the device functions it calls (warp_chol ... k_mid_solve)
                 "span": ("// Row of slot s owned by a lane in the warp-level factorization",
                          "// FP64 fallback of the precision form"),
                 "read_bytes": 427.399552e6, "write_bytes": 213.848576e6, "entries": 3774874, "slices": 8192}


def kernel_source_sha(rel_path: str, span=None) -> str:
    """sha256 prefix of a source file, or of the text between two markers."""
    import hashlib
    with open(os.path.join(ROOT, rel_path), "rb") as f:
        data = f.read()
    if span:
        txt = data.decode()
        a, b = txt.index(span[0]), txt.index(span[1])
        data = txt[a:b].encode()
    return hashlib.sha256(data).hexdigest()[:16]


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


# ------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ helpers

def als_flops_per_entry(r: int) -> int:
    """Algorithmic flops of one middle-level update per entry (Alg. 1):
    Hermitian Gram r^2(r^2+1)/2 + right-hand side r^2 complex multiply-adds,
    8 real flops each."""
    return 8 * (r * r * (r * r + 1) // 2 + r * r)


def max_over_ranks(x: float, dist_mod, device) -> float:
    """The largest value of x over all ranks (a job's step time is its slowest
    rank's); x itself when there is no process group."""
    if dist_mod is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, ms_step: float) -> float:
    """Whole-job units per second: every replica processes units_per_rank
    units per step of ms_step (the max over ranks)."""
    return world * units_per_rank / (ms_step * 1e-3)


def kernel_rooflines(prob, prof, stats, peaks, fp32_meas):
    """Per-kernel algorithmic work against the measured peaks (complex64
    precision form), from the library's CUDA-event timers of the timed sweeps.

    Bytes are what the algorithm must move through HBM per launch (complex64
    values of 8 bytes, 4-byte indices), flops are 8 per complex multiply-add
    of the algorithm's own operation count.  `frac` is against the measured
    copy bandwidth for the streaming kernels and the measured FP32 FMA peak
    for arithmetic."""
    n, L, r, nnz = prob.n, prob.L, prob.r, prob.nnz
    S = 1 << (L + 1)
    D = r * r
    npk = D * (D + 1) // 2
    hbm = peaks.get("hbm_gbs", 6800.0)
    slices = L * S * max(len(stats), 1)
    steps_avg = sum(int(st["refine_steps"]) for st in stats) / slices

    def avg_ms(key):
        cnt, tot = prof.get(key, (0, 0.0))
        return tot / cnt if cnt else None

    out = []
    ms = avg_ms("env_right")
    if ms:
        by = nnz * (16 * r + 4) + S * D * 8
        a = by / (ms * 1e-3) / 1e9
        out.append({"kernel": "k_env_right", "bound": "hbm", "launch_ms": ms, "bytes": by,
                    "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
                    "per_unit": f"{16 * r + 4} B per entry (w in, w out, level map) + {D * 8} B per slice"})
    ms = avg_ms("mid_solve")
    if ms:
        by = S * (npk + D) * 8 + nnz * (16 * r + 4) + S * D * 24 + 4 * (S + 1)
        fl = S * (4.0 / 3.0 * D ** 3 + 8.0 * D * D * (2 * (1 + steps_avg) + steps_avg)) + nnz * 8 * D
        a = by / (ms * 1e-3) / 1e9
        af = fl / (ms * 1e-3) / 1e12
        cap = SOLVE_TRAFFIC
        traffic = None
        if nnz == cap["entries"] and S == cap["slices"] and \
                kernel_source_sha(cap["source"], cap["span"]) == cap["sha"]:
            traffic = cap["read_bytes"] + cap["write_bytes"]
        out.append({"kernel": "k_mid_solve", "bound": "hbm", "launch_ms": ms, "bytes": by,
                    "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm, "traffic": traffic,
                    "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch at this "
                                      f"workload (kernel source sha {cap['sha']}: warp_chol through k_mid_solve)",
                    "flop": fl, "fp32_achieved_tflops": af, "fp32_peak": fp32_meas, "fp32_frac": af / fp32_meas,
                    "refine_steps_per_slice": steps_avg,
                    "per_unit": f"{(npk + D) * 8 + D * 24} B per slice (normal equations in, slice out) + "
                                f"{16 * r + 4} B per entry (h in, h out, level map); flop: complex Cholesky "
                                f"4/3 D^3, 8 D^2 per triangular solve pair and per residual, 8 r^2 per entry"})
    npo = r * (r + 1) // 2
    outer = [("outer_rows_gram", "k_outer_gram (rows)", nnz * (8 * r + 8) + n * (npo + r) * 16,
              f"{8 * r + 8} B per entry (w_0 row, value) + {(npo + r) * 16} B per row fiber (FP64 record)"),
             ("outer_cols_gram", "k_outer_gram (columns)", nnz * (8 * r + 8) + n * (npo + r) * 16,
              f"{8 * r + 8} B per entry (h_(L+1) row, value) + {(npo + r) * 16} B per column fiber"),
             ("outer_rows_post", "k_outer_post (rows)", nnz * (8 * r + 4) + n * r * 8,
              f"{8 * r + 4} B per entry (h_1 row written, level map) + {r * 8} B per fiber"),
             ("outer_cols_post", "k_outer_post (columns)", nnz * (8 * r + 8) + n * r * 8,
              f"{8 * r + 8} B per entry (h_(L+1) row, value) + {r * 8} B per fiber")]
    for key, name, by, unit in outer:
        ms = avg_ms(key)
        if ms:
            a = by / (ms * 1e-3) / 1e9
            out.append({"kernel": name, "bound": "hbm", "launch_ms": ms, "bytes": by, "achieved": a,
                        "peak": hbm, "unit": "GB/s", "frac": a / hbm, "per_unit": unit})
    ms = avg_ms("eval")
    if ms:
        nt = int(prob.it.size)
        fl = nt * 8 * (L * D + 2 * r)
        af = fl / (ms * 1e-3) / 1e12
        out.append({"kernel": "k_eval", "bound": "alu", "launch_ms": ms, "flop": fl,
                    "achieved": af, "peak": fp32_meas, "unit": "TFLOP/s", "frac": af / fp32_meas,
                    "per_unit": f"{8 * (L * D + 2 * r)} flop per test entry (L r x r complex products)",
                    "note": "thread per test entry; the slices come from L2 (factors fit in it)"})
    keymap = {"k_env_right": "env_right", "k_mid_solve": "mid_solve", "k_outer_gram (rows)": "outer_rows_gram",
              "k_outer_gram (columns)": "outer_cols_gram", "k_outer_post (rows)": "outer_rows_post",
              "k_outer_post (columns)": "outer_cols_post", "k_eval": "eval"}
    for o in out:
        o["ms_per_sweep"] = prof.get(keymap[o["kernel"]], (0, 0.0))[1] / max(len(stats), 1)
        o.setdefault("traffic", None)
    return out


def group_counts(prob):
    """Row / column groups of every middle level, by the library's rule:
    inside a slice of S^{m+1}, the entries of one row (levels with
    2m <= L + 1) or of one column share an environment."""
    pi, pj = prob.i.astype(np.int64) // prob.b, prob.j.astype(np.int64) // prob.b
    out = {}
    for m in range(1, prob.L + 1):
        k = ((pi >> (m - 1)) << m) | (pj >> (prob.L - m))
        by_col = 2 * m > prob.L + 1
        other = prob.j if by_col else prob.i
        out[m] = int(np.unique(k * prob.n + other).size)
    return out


def gram_rooflines(prob, prof, n_sweeps, c64, tc_levels, grouped, peaks, fp32_meas, fp64_meas, args):
    """Rooflines of the middle-level normal-equation kernels of the timed
    sweeps: the per-entry kernel (tensor cores, or CUDA cores) at the levels
    it ran, and the grouped CUDA-core kernel at the levels with few row /
    column groups (algorithmic flops: 8 (D(D+1)/2 + D) per group for the
    Kronecker updates plus 8 (r^2 + r) per entry for the group sums)."""
    r, nnz = prob.r, prob.nnz
    D = r * r
    out = []
    # grouped: {level: row / column groups} of the levels the library ran on
    # the grouped Gram (bfc_level_groups)
    n_plain = prob.L - len(grouped)
    cnt, tot = prof.get("mid_gram", (0, 0.0))
    if cnt and n_plain:
        ms = tot / cnt
        fl = nnz * als_flops_per_entry(r)
        a = fl / (ms * 1e-3) / 1e12
        if tc_levels:
            # tcgen05 kind::tf32: the measured sustained bf16 peak (the kernel
            # runs inside a long step) times the nominal dense TF32 / BF16
            # ratio 1.1 / 2.25
            peak = peaks.get("bf16_tflops_sustained", 1700.0) * 1.1 / 2.25
            executed = nnz * TC_FLOPS_PER_ENTRY / (ms * 1e-3) / 1e12
            traffic = None
            cap = TC_GRAM_TRAFFIC
            if not args.n and kernel_source_sha(cap["source"]) == cap["sha"]:
                traffic = (cap["read_bytes"] * nnz / cap["entries"]
                           + cap["write_bytes"] * (1 << (prob.L + 1)) / cap["slices"])
            out.append({"kernel": "k_mid_gram_tc", "bound": "tensor", "achieved": a, "peak": peak,
                        "unit": "TFLOP/s", "frac": a / peak, "traffic": traffic,
                        "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch at "
                                          f"n=32768 (kernel source sha {cap['sha']}), scaled by entries (reads) "
                                          "and slices (writes)",
                        "launch_ms": ms, "launches_per_sweep": n_plain, "ms_per_sweep": tot / n_sweeps,
                        "flop_per_launch": fl,
                        "per_unit": f"{als_flops_per_entry(r)} flop per entry (Hermitian Gram + right-hand side)",
                        "peak_source": "MEASURED_PEAKS bf16_tflops_sustained x 1.1/2.25 (of measured)",
                        "executed_tflops": executed, "executed_frac": executed / peak,
                        "executed_note": "issued MMA flops: 128 x 144 real embedding of the complex Gram "
                                         "(uu, uv, vu, vv full squares and the right-hand side, one contraction "
                                         "position per entry) x 3 TF32 split products = 110592 flop per entry",
                        "fp32_peak": fp32_meas, "fp32_frac": a / fp32_meas})
        else:
            peak = fp32_meas if c64 else fp64_meas
            out.append({"kernel": "k_mid_gram", "bound": "alu", "achieved": a, "peak": peak, "unit": "TFLOP/s",
                        "frac": a / peak, "traffic": None, "launch_ms": ms, "launches_per_sweep": n_plain,
                        "ms_per_sweep": tot / n_sweeps, "flop_per_launch": fl,
                        "per_unit": f"{als_flops_per_entry(r)} flop per entry",
                        "peak_source": ("measured FP32" if c64 else "measured FP64") +
                                       " FMA-chain peak (bfc_measure_alu_peaks, of measured)"})
    cnt, tot = prof.get("mid_gram_grp", (0, 0.0))
    if cnt and grouped:
        # one profiling scope per grouped level covers its two kernels (group
        # sums, then the per-slice Kronecker updates)
        ms = tot / (n_sweeps * len(grouped))
        per_group = 8 * (D * (D + 1) // 2 + D)
        per_entry = 8 * (D + r)
        fl = (sum(grouped.values()) * per_group + len(grouped) * nnz * per_entry) / len(grouped)
        a = fl / (ms * 1e-3) / 1e12
        peak = fp32_meas if c64 else fp64_meas
        out.append({"kernel": "k_group_sums + k_mid_gram_grp", "bound": "alu", "achieved": a, "peak": peak, "unit": "TFLOP/s",
                    "frac": a / peak, "traffic": None, "launch_ms": ms, "launches_per_sweep": len(grouped),
                    "ms_per_sweep": tot / n_sweeps, "flop_per_launch": fl,
                    "groups_per_level": grouped,
                    "per_unit": f"{per_group} flop per row / column group (Kronecker update of the Hermitian "
                                f"Gram + right-hand side) + {per_entry} flop per entry (group sums)",
                    "peak_source": ("measured FP32" if c64 else "measured FP64") +
                                   " FMA-chain peak (bfc_measure_alu_peaks, of measured)",
                    "per_entry_equivalent_tflops": nnz * als_flops_per_entry(r) / (ms * 1e-3) / 1e12})
    return out


def lowrank_start(prob, bfc_mod, prec, gram=0, group_ratio=0.0):
    import synth
    A0, B0 = synth.random_lowrank_start(prob, prob.r)
    c = bfc_mod.Completion(prob.n, prob.L, prob.b, prob.r, prob.lam, prob.i, prob.j, prob.t,
                           prob.it, prob.jt, prob.tt, prec=prec, gram_impl=gram, group_ratio=group_ratio)
    c.lowrank_init(A0, B0, 10)
    return c


def time_to_tolerance(bfc_mod, prec, tol=1e-3, max_sweeps=30):
    """Full workflow (Sec. 4.3) at n = 65536 with the paper's sampling rule
    |Omega| = 6 r n log2 n (Sec. 5.1; r = 8): low-rank start on the GPU, then
    ALS sweeps until the relative test error (Eq. BF_convergence on the
    held-out entries) is below tol.  Returns seconds (wall, from the start of
    the low-rank completion), sweeps and the error trajectory."""
    import synth
    n, L, b, r = 65536, 12, 16, 8
    prob = synth.make_problem("n65536_paper_sampling", n, L, b, r, math.pi * n / 16, 1.5,
                              6 * r * n * 16, 1e-7, max_sweeps, synth.SEED_BASE + 16 * 3)
    A0, B0 = synth.random_lowrank_start(prob, r)
    c = bfc_mod.Completion(n, L, b, r, prob.lam, prob.i, prob.j, prob.t, prob.it, prob.jt, prob.tt,
                           prec=prec)
    t0 = time.perf_counter()
    c.lowrank_init(A0, B0, 10)
    errs, reached = [], None
    for s in range(max_sweeps):
        st = c.sweep()
        errs.append(st["test_rel_err"])
        if st["test_rel_err"] < tol:
            reached = time.perf_counter() - t0
            break
    total = time.perf_counter() - t0
    c.close()
    return {"seconds": reached, "sweeps": len(errs) if reached else None, "wall_s": total,
            "nnz_train": prob.nnz, "test_rel_err": [float(f"{e:.3e}") for e in errs]}


def run_config_table(bfc_mod, tol=1e-3):
    """The small single-problem configurations (n = 256: plain ALS, 10
    sweeps; n = 4096 with 1e-4 noise: ALS, 20 sweeps, and L-BFGS, 200
    iterations) for the plain FP64 path and the precision form: ms per
    sweep (library CUDA events), entries/s, time to test error tol (wall,
    from the start of the low-rank completion, 10 sweeps of Alg. 1 with
    L = 0), final test error; and the oracle's whole sweep on one host
    thread and on all of them."""
    import oracle
    import synth
    oracle.build()
    cores = host_cores()
    out = {}
    for k, iters in ((1, 10), (2, 20)):
        p = synth.config(k)
        A0, B0 = synth.random_lowrank_start(p, p.r)
        row = {"workload": f"n={p.n} L={p.L} b={p.b} r={p.r}, {p.nnz} train entries", "nnz_train": p.nnz}
        X0 = None
        for name, prec in (("plain_fp64", bfc_mod.PREC_FP64), ("precision_form", bfc_mod.PREC_C64)):
            c = bfc_mod.Completion(p.n, p.L, p.b, p.r, p.lam, p.i, p.j, p.t, p.it, p.jt, p.tt, prec=prec)
            try:
                t0 = time.perf_counter()
                c.lowrank_init(A0, B0, 10)
                if X0 is None:
                    X0 = c.get_factors()
                errs, ms, reached = [], [], None
                for _ in range(iters):
                    st = c.sweep()
                    errs.append(st["test_rel_err"])
                    ms.append(st["sweep_ms"])
                    if reached is None and st["test_rel_err"] < tol:
                        reached = time.perf_counter() - t0
                med = float(np.median(ms))
                row[name] = {"ms_per_sweep": med, "entries_per_s": p.nnz / (med * 1e-3),
                             "seconds_to_tol": reached, "final_test_rel_err": errs[-1],
                             "test_rel_err": [float(f"{e:.3e}") for e in errs]}
            finally:
                c.close()
        if k == 2:
            for name, prec in (("lbfgs_plain_fp64", bfc_mod.PREC_FP64), ("lbfgs_precision_form", bfc_mod.PREC_C64)):
                c = bfc_mod.Completion(p.n, p.L, p.b, p.r, p.lam, p.i, p.j, p.t, p.it, p.jt, p.tt, prec=prec)
                try:
                    t0 = time.perf_counter()
                    c.lowrank_init(A0, B0, 10)
                    hist = c.lbfgs(200)
                    wall = time.perf_counter() - t0
                    te = [h["test_rel_err"] for h in hist]
                    row[name] = {"iterations": len(hist), "seconds": wall, "final_test_rel_err": te[-1],
                                 "best_test_rel_err": min(te)}
                finally:
                    c.close()
        m1, t1 = time_oracle_sweep(p, X0, 1, threads=1)
        mall, tall = time_oracle_sweep(p, X0, 1, threads=cores)
        row["cpu_oracle"] = {"serial_s_per_sweep": t1, "all_cores_s_per_sweep": tall, "cores": cores}
        out[f"config{k}"] = row
    return out


def oracle_sample(prob, frac_every: int):
    """Every `frac_every`-th training entry of the workload."""
    sel = np.arange(0, prob.nnz, frac_every)
    return prob.i[sel], prob.j[sel], prob.t[sel]


def run_batched(bfc_mod, count=64, max_sweeps=20, tol=1e-4):
    """The batched workload (64 independent problems, n in 1024..16384,
    r in {4, 6, 8}, |Omega| = c n log2 n, c in [4, 8]) in the precision form
    through bfc_batch_complete: low-rank starts, the per-rank Gram autotuning,
    then every remaining sweep of every problem in one graph launch (a
    conditional loop per problem that stops at its training tolerance or
    max_sweeps)."""
    import synth
    probs = synth.batch_problems(count)
    cs = [bfc_mod.Completion(p.n, p.L, p.b, p.r, p.lam, p.i, p.j, p.t, p.it, p.jt, p.tt,
                             prec=bfc_mod.PREC_C64, max_sweeps=max_sweeps, tol=tol,
                             seed=synth.BATCH_SEED_BASE + 16 * q + synth.SEED_INIT,
                             init_kind=1, lr_sweeps=10)
          for q, p in enumerate(probs)]
    try:
        t0 = time.perf_counter()
        last = bfc_mod.batch_complete(cs)
        wall = time.perf_counter() - t0
    finally:
        for c in cs:
            c.close()
    sweeps = [st["sweep"] for st in last]
    entry_sweeps = sum(p.nnz * s for p, s in zip(probs, sweeps))
    gram = {}
    for p, st in zip(probs, last):
        gram[str(p.r)] = "tensor" if st["gram_impl"] == 0 else "cuda"
    test = sorted(st["test_rel_err"] for st in last)
    versus = batch_vs_fp64(bfc_mod)
    return {"vs_plain_fp64": versus,
            "workload": f"{count} problems, n in 1024..16384, r in {{4,6,8}}, |Omega| = c n log2 n, "
                        "c in [4,8], precision form, low-rank start (10 sweeps), tol 1e-4 train",
            "problems": count, "entries_total": int(sum(p.nnz for p in probs)),
            "sweeps_total": int(sum(sweeps)), "seconds": wall,
            "entry_sweeps_per_s": entry_sweeps / wall,
            "gram_kernel_by_rank": gram,
            "test_rel_err_median": test[len(test) // 2], "test_rel_err_max": test[-1]}


def batch_vs_fp64(bfc_mod, count=16, max_sweeps=30, tol_train=5e-4):
    """Time for a batch of problems to reach test error 1e-3, three arms from
    the same low-rank starts and with the same stop rule (training error
    below tol_train, at which these noise-free problems' test errors are
    below 1e-3; the count that made it is reported per arm):
      batched   the precision form through bfc_batch_complete (all sweeps in
                one graph launch after the per-rank autotuning);
      sequential the same precision form, problem by problem (bfc_complete):
                the gain of batching itself;
      plain_fp64 FP64 ALS problem by problem (bfc_complete).
    Problems: n in {1024, 2048, 4096}, r in {4, 6, 8}, the cfg-4 operator
    family with the paper's sampling rule 6 r n log2 n (the c n log2 n,
    c in [4, 8] draws are information-limited)."""
    import synth
    probs = synth.batch_problems(count, seed_base=synth.BATCH_SEED_BASE + 0x8000,
                                 n_choices=(1024, 2048, 4096), paper_rule=True)

    def make(p, prec, q):
        return bfc_mod.Completion(p.n, p.L, p.b, p.r, p.lam, p.i, p.j, p.t, p.it, p.jt, p.tt, prec=prec,
                                  max_sweeps=max_sweeps, tol=tol_train, seed=4242 + q,
                                  init_kind=1, lr_sweeps=10)

    def summary(last, seconds):
        te = [st["test_rel_err"] for st in last]
        return {"seconds": seconds, "test_err_below_1e-3": int(sum(e < 1e-3 for e in te)),
                "test_err_median": float(np.median(te)), "test_err_max": float(np.max(te)),
                "sweeps_median": float(np.median([st["sweep"] for st in last]))}

    cs = [make(p, bfc_mod.PREC_C64, q) for q, p in enumerate(probs)]
    try:
        t0 = time.perf_counter()
        last = bfc_mod.batch_complete(cs)   # synchronous
        t_batch = time.perf_counter() - t0
    finally:
        for c in cs:
            c.close()
    arms = {"batched": summary(last, t_batch)}
    arms["batched"]["graph_launches_after_autotune"] = int(max(st["batch_launches"] for st in last))
    for name, prec in (("sequential", bfc_mod.PREC_C64), ("plain_fp64", bfc_mod.PREC_FP64)):
        t, lst = 0.0, []
        for q, p in enumerate(probs):
            c = make(p, prec, q)
            try:
                t0 = time.perf_counter()
                lst.append(c.complete()[-1])
                t += time.perf_counter() - t0
            finally:
                c.close()
        arms[name] = summary(lst, t)
    return {"problems": count, "entries_total": int(sum(p.nnz for p in probs)),
            "stop": f"training error < {tol_train} or {max_sweeps} sweeps (every arm); no FP64 refinement sweeps",
            "arms": arms,
            "speedup_vs_plain_fp64": arms["plain_fp64"]["seconds"] / arms["batched"]["seconds"],
            "speedup_of_batching": arms["sequential"]["seconds"] / arms["batched"]["seconds"]}


def run_learned(bfc_mod, n_train=64, n_test=8, epochs=2500, max_sweeps=30, tol=1e-3, c_obs=36, with_nn=False):
    """The learned-start workload: family n = 4096, L = 8, b = 16, r = 6,
    omega / (pi n) ~ U[1/16, 1/4], h ~ U[0.5, 2], |Omega| = c_obs n log2 n
    at the same sample positions for every member, lambda = 1e-7 (c_obs = 36
    is the paper's 6 r n log n rule; 6 n log n leaves the family
    information-limited: no held-out draw falls below test error 1).  Training:
    n_train precision-form completions (fixed-seed low-rank start, 15 sweeps,
    run as batches through bfc_batch_complete), gauge-fixed by
    bfc_canonicalize, then the MLP 2 -> 256 -> 256 -> 2P trained by
    bfc_mlp_train.  Held-out draws: ALS from the learned start (precision
    form) against the low-rank start in the precision form and in plain
    FP64, up to max_sweeps sweeps or test error < tol."""
    import synth
    n, L, b, r = 4096, 8, 16, 6
    nobs = c_obs * n * 12
    base = synth.BATCH_SEED_BASE + 0x10000
    rng = synth.SplitMix64(base + synth.SEED_PARAMS)

    shared = {}

    def problem(q):
        u = rng.uniform(2)
        om, h = 1 / 16 + u[0] * (1 / 4 - 1 / 16), 0.5 + 1.5 * u[1]
        if "base" not in shared:   # the sample positions, drawn once for the family
            shared["base"] = synth.make_problem(f"learned{q}", n, L, b, r, om * math.pi * n, h, nobs, 1e-7, 15,
                                                base)
            return om, h, shared["base"]
        return om, h, synth.family_member(shared["base"], f"learned{q}", om * math.pi * n, h)

    def completion(p, prec, **kw):
        return bfc_mod.Completion(p.n, p.L, p.b, p.r, p.lam, p.i, p.j, p.t, p.it, p.jt, p.tt, prec=prec, **kw)

    t0 = time.perf_counter()
    X, Y = [], []
    for c0 in range(0, n_train, 32):
        group = [problem(c0 + q) for q in range(min(32, n_train - c0))]
        cs = [completion(p, bfc_mod.PREC_C64, init_kind=1, seed=777, max_sweeps=15, tol=1e-12, lr_sweeps=10)
              for _, _, p in group]
        try:
            bfc_mod.batch_complete(cs)
            for (om, h, _), c in zip(group, cs):
                c.canonicalize()
                X.append((om, h))
                Y.append(c.get_factors().view(np.float64).copy())
        finally:
            for c in cs:
                c.close()
    t_data = time.perf_counter() - t0
    X, Y = np.array(X), np.array(Y)
    t0 = time.perf_counter()
    model = bfc_mod.Mlp(2, 256, Y.shape[1], seed=5)
    hist = bfc_mod.bfc_mlp_train(model.h, X, Y, epochs=epochs, batch=32, lr=1e-3, seed=3)
    t_train = time.perf_counter() - t0
    if not with_nn:
        del Y

    def run(p, start, prec):
        c = completion(p, prec, init_kind=1 if start == "lowrank" else 0, seed=777, max_sweeps=0, lr_sweeps=10)
        try:
            t1 = time.perf_counter()
            if start == "learned":
                bfc_mod.bfc_init_learned(c.ctx, model.h, p.omega, p.h, allow_fallback=False)
            elif start == "nearest":
                om = p.omega / (math.pi * n)
                k = int(np.argmin(((X[:, 0] - om) / 0.1875) ** 2 + ((X[:, 1] - p.h) / 1.5) ** 2))
                c.set_factors(Y[k].view(np.complex128))
            else:
                c.complete()
            errs, reached = [], None
            for s in range(max_sweeps):
                st = c.sweep()
                errs.append(st["test_rel_err"])
                if st["test_rel_err"] < tol:
                    reached = time.perf_counter() - t1
                    break
            return errs, reached
        finally:
            c.close()

    out = {"learned_pc64": [], "lowrank_pc64": [], "lowrank_fp64": [], "nearest_pc64": []}
    for q in range(n_test):
        _, _, p = problem(10000 + q)
        out["learned_pc64"].append(run(p, "learned", bfc_mod.PREC_C64))
        if with_nn:
            out["nearest_pc64"].append(run(p, "nearest", bfc_mod.PREC_C64))
        out["lowrank_pc64"].append(run(p, "lowrank", bfc_mod.PREC_C64))
        out["lowrank_fp64"].append(run(p, "lowrank", bfc_mod.PREC_FP64))
    model.close()

    def summary(rs):
        e1 = [e[0] for e, _ in rs]
        e5 = [e[min(4, len(e) - 1)] for e, _ in rs]
        last = [e[-1] for e, _ in rs]
        t = [x for _, x in rs if x is not None]
        return {"test_err_after_1_sweep_median": float(np.median(e1)),
                "test_err_after_5_sweeps_median": float(np.median(e5)),
                "best_test_err_median": float(np.median([min(e) for e, _ in rs])),
                "final_test_err_median": float(np.median(last)),
                "reached_tol": f"{len(t)}/{len(rs)}",
                "seconds_to_tol_median": float(np.median(t)) if t else None}

    res = {"workload": f"n=4096 L=8 b=16 r=6 family, omega/(pi n) in [1/16,1/4], h in [0.5,2], "
                        f"|Omega|={c_obs} n log2 n (shared positions); {n_train} training completions, "
                        f"{n_test} held-out draws, tol {tol} test error, <= {max_sweeps} sweeps",
            "training_data_seconds": t_data, "mlp_train_seconds": t_train,
            "mlp_loss_first_last": [float(hist[0]), float(hist[-1])],
            "learned_start_precision_form": summary(out["learned_pc64"]),
            "lowrank_start_precision_form": summary(out["lowrank_pc64"]),
            "lowrank_start_plain_fp64": summary(out["lowrank_fp64"])}
    if with_nn:
        res["nearest_training_completion_start"] = summary(out["nearest_pc64"])
    return res


def run_first_order(bfc_mod, c, prob, hbm_peak, iters=3, nvec=64):
    """The first-order methods and the matrix-vector product on the bench
    workload, from the context's current factors: `iters` iterations of ADAM
    (Alg. 3/4, alpha 1e-3) and of ADF (Alg. 5 with the App. A.3 sweeps), and
    U = X(S) V for nvec vectors (Eq. butterfly-mat-vec), each timed by the
    library's per-kernel CUDA events."""
    X0 = c.get_factors()
    out = {}
    for name, run in (("adam", lambda: c.adam(iters, alpha=1e-3)), ("adf", lambda: c.adf(iters))):
        c.set_factors(X0)
        c.profile(True)
        hist = run()
        prof = c.profile_read()
        c.profile(False)
        ms = sum(v[1] for v in prof.values()) / iters
        out[name] = {"ms_per_iter": ms, "entries_per_s": prob.nnz / (ms * 1e-3),
                     "train_rel_err": [float(f"{h['train_rel_err']:.4e}") for h in hist],
                     "kernels_ms": {k: round(v[1] / iters, 4) for k, v in prof.items()}}
    c.set_factors(X0)
    V = np.zeros((prob.n, nvec), dtype=np.complex128)
    V.real = np.random.default_rng(0).standard_normal((prob.n, nvec))
    c.matvec(V)   # warm-up
    c.profile(True)
    c.matvec(V)
    prof = c.profile_read()
    c.profile(False)
    ms = sum(v[1] for v in prof.values())
    vsz = 8 if c.params.prec == bfc_mod.PREC_C64 else 16
    fbytes = c.P * vsz
    # the level-by-level contraction streams its intermediates: per vector,
    # the leaf writes n/b r-vectors, every middle level reads two children and
    # writes one r-vector per slice, the root reads two per leaf block
    r, L, S, nb = prob.r, prob.L, 1 << (prob.L + 1), prob.n // prob.b
    inter = nvec * r * vsz * (nb + (L - 1) * 3 * S + 2 * S + 2 * nb)
    by = fbytes + 2 * prob.n * nvec * 16 + inter
    out["matvec"] = {"nvec": nvec, "kernel_ms": ms, "vectors_per_s": nvec / (ms * 1e-3),
                     "kernels_ms": {k: round(v[1], 4) for k, v in prof.items()},
                     "roofline": {"bound": "hbm", "bytes": by, "achieved": by / (ms * 1e-3) / 1e9,
                                  "peak": hbm_peak, "unit": "GB/s", "frac": by / (ms * 1e-3) / 1e9 / hbm_peak,
                                  "per_unit": "all factors once (compute type) + 16 B per vector entry in and out + "
                                              "the level intermediates (r values per slice and vector: the leaf "
                                              "writes n/b, each middle level reads 2 S and writes S, the root "
                                              "reads 2 n/b)",
                                  "flop": 8 * nvec * (prob.n * r + L * S * r * r + prob.n * r)}}
    return out


def run_radon(bfc_mod, sweeps=20, fp64_sweeps=2, init_kind=1, lr_rank=0):
    """The Radon-transform workload of Sec. 5.3 at the paper's convergence
    study: n = 4096, leaf size 4 (L = 10), rank estimate 12, 3,440,640
    training and 491,520 test entries (7 r n log2 n and r n log2 n with the
    actual rank 10), lambda = 1e-8; the low-rank start of rank r (10 sweeps
    of Alg. 1 with L = 0, exact embedding; a start of lower rank would leave
    the extra rank directions at zero, where ALS never moves them); then ALS
    sweeps in the precision form, and the first sweeps in plain FP64 on the
    same GPU for the time per sweep."""
    import synth
    p = synth.radon_problem(sweeps=sweeps)
    out = {"workload": f"radon n={p.n} L={p.L} b={p.b} r={p.r}, |Omega| = 70 n log2 n ({p.nnz} train / "
                       f"{p.it.size} test), lambda=1e-8, start: rank-{lr_rank or p.r} low-rank completion "
                       f"(10 sweeps), {'Alg. 2 conversion' if init_kind == 2 else 'exact embedding'}"}
    for name, prec, ns in (("precision_form", bfc_mod.PREC_C64, sweeps), ("plain_fp64", bfc_mod.PREC_FP64,
                                                                          fp64_sweeps)):
        c = bfc_mod.Completion(p.n, p.L, p.b, p.r, p.lam, p.i, p.j, p.t, p.it, p.jt, p.tt, prec=prec,
                               max_sweeps=ns, tol=1e-12, seed=p.seed + synth.SEED_INIT, init_kind=init_kind,
                               lr_rank=lr_rank, lr_sweeps=10)
        try:
            t0 = time.perf_counter()
            hist = c.complete()
            wall = time.perf_counter() - t0
        finally:
            c.close()
        te = [h["test_rel_err"] for h in hist]
        tr = [h["train_rel_err"] for h in hist]
        out[name] = {"sweeps": len(hist), "seconds_with_start": wall,
                     "ms_per_sweep": float(np.median([h["sweep_ms"] for h in hist])),
                     "test_rel_err": [float(f"{e:.3e}") for e in te],
                     "train_rel_err": [float(f"{e:.3e}") for e in tr],
                     "first_sweep_train_below_1e-3": next((q + 1 for q, e in enumerate(tr) if e < 1e-3), None),
                     "first_sweep_test_below_1e-3": next((q + 1 for q, e in enumerate(te) if e < 1e-3), None)}
    return out


def time_oracle_sweep(prob, X0, frac_every: int, threads: int = 1):
    """One oracle ALS sweep over every frac_every-th training entry (1 = all
    of them) on `threads` host threads; returns (entries, seconds)."""
    import oracle
    i, j, t = oracle_sample(prob, frac_every)
    with oracle.threads(threads):
        t0 = time.perf_counter()
        oracle.als_sweep(prob.n, prob.L, prob.b, prob.r, prob.lam, X0, i, j, t)
        dt = time.perf_counter() - t0
    return len(i), dt


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline_line(prob, X0):
    """The oracle on the host: one whole ALS sweep of every training entry on
    all cores (the OpenMP variant, bit-identical to the serial oracle), and
    the serial oracle over 1 % and 2 % samples fitted to a whole sweep."""
    cores = host_cores()
    mall, tall = time_oracle_sweep(prob, X0, 1, threads=cores)
    m1, t1 = time_oracle_sweep(prob, X0, 100)
    m2, t2 = time_oracle_sweep(prob, X0, 50)
    v1, t_full = oracle_full_rate(prob, m1, t1, m2, t2)
    return {"value": mall / tall, "unit": UNIT, "cores": cores, "kind": "oracle", "nproc": cores,
            "sample": f"one whole oracle ALS sweep of all {mall} training entries at the full n=65536 L=12 r=8 "
                      f"shape on {cores} host threads ({tall:.1f} s; OpenMP over independent systems and "
                      "entries, bit-identical to the serial oracle)",
            "serial": {"value": v1, "unit": UNIT, "cores": 1,
                       "sample": oracle_sample_text(m1, t1, m2, t2, t_full)}}


def oracle_full_rate(prob, m1, t1, m2, t2):
    """Fit t = a + b m to two sampled sweeps (a: the per-slice and per-fiber
    solves, which a sample keeps in full; b: per-entry work) and return the
    entries/s of a full sweep over all training entries."""
    b = max((t2 - t1) / max(m2 - m1, 1), 1e-12)
    a = max(t1 - b * m1, 0.0)
    t_full = a + b * prob.nnz
    return prob.nnz / t_full, t_full


def oracle_sample_text(m1, t1, m2, t2, t_full):
    return (f"oracle ALS sweeps at the full n=65536 L=12 r=8 shape over 1% ({m1} entries, {t1:.1f} s) and "
            f"2% ({m2} entries, {t2:.1f} s) of the training entries; t = a + b*entries fitted to the two "
            f"and extrapolated to all 3774874 entries ({t_full:.0f} s per sweep)")


# ------------------------------------------------------------ reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    import synth
    oracle.build()
    prob = synth.config(3)
    X0 = synth.random_factors(prob.n, prob.L, prob.r, prob.seed + synth.SEED_PLANT, sigma=0.3)
    cores = host_cores()
    # each step: the oracle (OpenMP variant, all host cores) sweeps every
    # stride-th training entry at the full shape, all slices and fibers
    # solved; the stride (4 up to 15 steps, larger beyond) keeps the whole run
    # to a few minutes; warm-up steps sweep 1 %
    stride = 4 * max(1, -(-args.steps // 15))
    for _ in range(args.warmup):
        time_oracle_sweep(prob, X0, 100, threads=cores)
    times = []
    m = 0
    for _ in range(args.steps):
        m, dt = time_oracle_sweep(prob, X0, stride, threads=cores)
        times.append(dt)
    t_step = statistics.mean(times)
    value = m / t_step
    sample = (f"each step: one oracle ALS sweep (complex128, OpenMP variant on {cores} host threads, "
              f"bit-identical to the serial oracle) over every {stride}th training entry ({m} entries) at the full "
              f"n=65536 L=12 r=8 shape, all 98304 slice and 131072 fiber systems solved; {t_step:.2f} s per "
              "step; warm-up steps sweep 1 %")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": f"host, {cores} threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ our arm

def run_bfc(args, rank, world, local_rank):
    import torch

    import paper_2510_17734_gb300 as bfc
    import synth

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    bfc.load()
    dist = None
    if world > 1:
        import torch.distributed as dist
    prob = synth.config(3, n_override=args.n or None)
    workload = WORKLOAD if not args.n else (
        f"n={prob.n} L={prob.L} b={prob.b} r={prob.r}, the n=65536 construction at reduced n "
        f"(profiling case, {prob.nnz} train entries)")
    prec = bfc.PREC_C64 if args.prec == "c64" else bfc.PREC_FP64

    c = lowrank_start(prob, bfc, prec, gram={"auto": bfc.GRAM_AUTO, "tensor": bfc.GRAM_TENSOR,
                                             "cuda": bfc.GRAM_CUDA}[args.gram], group_ratio=args.group_ratio)
    stream = torch.cuda.Stream(device=dev)
    bfc.bfc_set_stream(c.ctx, stream.cuda_stream)

    for _ in range(args.warmup):
        c.sweep()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    stats = []
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            stats.append(c.sweep())
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_total = ev0.elapsed_time(ev1)
    ms_step = ms_total / args.steps
    # per-kernel times: the same number of sweeps again with the library's
    # per-kernel CUDA events on (kernels launched one by one, not from the
    # captured sweep graph the timed sweeps replay)
    c.profile(True)
    for _ in range(args.steps):
        c.sweep()
    prof = c.profile_read()
    c.profile(False)
    ms_step = max_over_ranks(ms_step, dist, dev)
    value = job_throughput(prob.nnz, world, ms_step)

    # end to end through the public API with host buffers (pinned)
    P = c.P
    host_in = torch.empty(2 * P, dtype=torch.float64, pin_memory=True)
    host_out = torch.empty(2 * P, dtype=torch.float64, pin_memory=True)
    host_in.copy_(torch.from_numpy(c.get_factors().view(np.float64)))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        bfc.bfc_set_factors(c.ctx, host_in)
        bfc.bfc_als_sweep(c.ctx)
        bfc.bfc_get_factors(c.ctx, host_out)
    torch.cuda.synchronize()
    e2e_ms = 1e3 * (time.perf_counter() - t0) / args.steps
    e2e_ms = max_over_ranks(e2e_ms, dist, dev)
    e2e_value = job_throughput(prob.nnz, world, e2e_ms)

    # gradient sweep (Eqs. (grad_butterfly_1), (grad_butterfly_l),
    # (grad_butterfly_last)): the full gradient of the regularized objective
    # on the device (bfc_grad with no host copy), kernels timed by the
    # library's CUDA events, the call by the host clock
    for _ in range(2):
        bfc.bfc_grad(c.ctx, True)
    ng = 5
    c.profile(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ng):
        bfc.bfc_grad(c.ctx, True)
    torch.cuda.synchronize()
    grad_wall_ms = 1e3 * (time.perf_counter() - t0) / ng
    gprof = c.profile_read()
    c.profile(False)
    grad_ms = sum(v[1] for v in gprof.values()) / ng
    gm_n, gm_ms = gprof.get("grad_mid", (0, 0.0))
    grad_mid_roof = None
    if gm_n:
        r_, S_ = prob.r, 1 << (prob.L + 1)
        by = prob.nnz * (24 * r_ + 20) + S_ * r_ * r_ * 24
        a = by / (gm_ms / gm_n * 1e-3) / 1e9
        hbm_peak = load_peaks().get("hbm_gbs", 6800.0)
        grad_mid_roof = {"kernel": "k_grad_mid", "bound": "hbm", "launch_ms": gm_ms / gm_n, "bytes": by,
                         "achieved": a, "peak": hbm_peak, "unit": "GB/s", "frac": a / hbm_peak,
                         "per_unit": f"{24 * r_ + 20} B per entry (h in and out, w, r in and out, level map) + "
                                     f"{r_ * r_ * 24} B per slice (Z in, gradient out)"}
    gradient = {"kernel_ms": grad_ms, "call_ms": grad_wall_ms, "roofline_grad_mid": grad_mid_roof,
                "entries_per_s": world * prob.nnz / (grad_ms * 1e-3),
                "kernels_ms": {k: round(v[1] / ng, 4) for k, v in gprof.items()},
                "note": "one full gradient (all factors) per call, device-resident; call_ms includes the "
                        "host synchronisation for the objective"}

    # rooflines of the normal-equation kernels and of the others; the line's
    # "roofline" is the kernel with the most device time per sweep
    launches = sum(int(st["launches"]) for st in stats)   # kernels launched by the timed sweeps
    clocks = clk.summary()
    peaks = load_peaks()
    fp32_meas, fp64_meas = bfc.bfc_measure_alu_peaks()
    n_sweeps = max(args.steps, 1)
    tc_levels = prec == bfc.PREC_C64 and args.gram != "cuda" and prob.r <= 8
    grouped = {}
    for m in range(1, prob.L + 1):
        ng, on = c.level_groups(m)
        if on:
            grouped[m] = ng
    entries = gram_rooflines(prob, prof, n_sweeps, prec == bfc.PREC_C64, tc_levels, grouped,
                             peaks, fp32_meas, fp64_meas, args)
    entries += kernel_rooflines(prob, prof, stats, peaks, fp32_meas) if prec == bfc.PREC_C64 else []
    if not entries:
        raise RuntimeError(f"no kernel timings in the profile: {sorted(prof)}")
    roofline = dict(max(entries, key=lambda x: x["ms_per_sweep"]))
    kernel_roof = entries
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64+f64" if prec == bfc.PREC_C64 else "f64",
            "data": "synthetic",
            "config": {"workload": workload, "precision": args.prec, "gram": args.gram,
                       "grouped_levels": sorted(grouped),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "working set > L2 (no flush)", "nnz_train": prob.nnz},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 16 * P,
                    "d2h_bytes_per_step": 16 * P + 64, "ms_per_step": e2e_ms},
            "gpu_launches": launches,
            "kernels_ms": {k: round(v[1] / max(args.steps, 1), 4) for k, v in prof.items()},
            "roofline": roofline,
            "kernel_rooflines": kernel_roof,
            "gradient": gradient,
            "alu_peaks_measured": {"fp32_tflops": fp32_meas, "fp64_tflops": fp64_meas,
                                   "how": "bfc_measure_alu_peaks: dependent FMA chains on all SMs, best of 5"},
            "clocks": clocks,
            "sweep_stats": {"train_rel_err": stats[-1]["train_rel_err"],
                            "test_rel_err": stats[-1]["test_rel_err"],
                            "fp64_fallback_fraction": (sum(int(st["refined_fallbacks"]) for st in stats)
                                                       / (len(stats) * prob.L * (1 << (prob.L + 1)))),
                            "refine_steps_per_slice": (sum(int(st["refine_steps"]) for st in stats)
                                                       / (len(stats) * prob.L * (1 << (prob.L + 1))))}}

    if not args.no_first_order:
        X_keep = c.get_factors()
        line["first_order"] = run_first_order(bfc, c, prob, load_peaks().get("hbm_gbs", 6800.0))
        c.set_factors(X_keep)
    if not args.no_radon and not args.n:
        line["radon"] = run_radon(bfc)

    if not args.no_ttt:
        # the specified workload cannot generalize (|Omega| = 4 n log2 n gives about one
        # observation per free parameter): report its best test error, and time to 1e-3
        # on the same operator with the paper's sampling rule, precision form and FP64
        best = min(h["test_rel_err"] for h in stats)
        ttt_c64 = time_to_tolerance(bfc, bfc.PREC_C64)
        ttt_f64 = time_to_tolerance(bfc, bfc.PREC_FP64, max_sweeps=8)
        line["time_to_1e-3_test_error"] = {
            "workload": "same operator, |Omega| = 6 r n log2 n = 48 n log2 n (paper's rule), lambda=1e-7",
            "precision_form": ttt_c64, "plain_fp64": ttt_f64,
            "speedup_vs_fp64": (ttt_f64["seconds"] / ttt_c64["seconds"]
                                if ttt_c64["seconds"] and ttt_f64["seconds"] else None),
            "specified_workload_best_test_rel_err": best,
            "specified_workload_note": "|Omega| = 4 n log2 n: test error does not fall below 1 (information limit)"}

    if not args.no_batch and not args.n:
        line["batched"] = run_batched(bfc)
    if not args.no_learned and not args.n:
        line["learned_start"] = run_learned(bfc, n_train=args.learned_train, n_test=args.learned_test,
                                            epochs=args.learned_epochs)

    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        X0 = c.get_factors()
        line["cpu_baseline"] = cpu_baseline_line(prob, X0)
    c.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)   # about 1 s timed: several clock samples at 200 ms
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="bfc", choices=["bfc", "reference"])
    ap.add_argument("--prec", default="c64", choices=["c64", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-tolerance runs")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-workload run")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-start run")
    ap.add_argument("--no-first-order", action="store_true", help="skip the ADAM / ADF / matvec run")
    ap.add_argument("--no-radon", action="store_true", help="skip the Radon-transform run")
    ap.add_argument("--learned-train", type=int, default=64, help="training completions of the learned start")
    ap.add_argument("--learned-epochs", type=int, default=2500, help="training epochs of the learned start")
    ap.add_argument("--learned-test", type=int, default=8, help="held-out draws of the learned start")
    ap.add_argument("--configs-table", action="store_true",
                    help="measure the n = 256 and n = 4096 configurations (GPU both paths, L-BFGS, oracle) and "
                         "print their JSON")
    ap.add_argument("--learned-only", action="store_true",
                    help="run only the learned-start experiment (its sizes from the --learned-* flags) and print "
                         "its JSON")
    ap.add_argument("--group-ratio", type=float, default=0.0,
                    help="groups-per-entry threshold of the grouped Gram (0: library default, < 0: never)")
    ap.add_argument("--gram", default="auto", choices=["auto", "tensor", "cuda"],
                    help="middle-level Gram: auto (grouped CUDA-core kernel at levels with few row / column "
                         "groups, tcgen05 per entry elsewhere), tensor (tcgen05 per entry), cuda (CUDA cores "
                         "per entry)")
    ap.add_argument("--n", type=int, default=0,
                    help="reduced n with the same construction (small profiling captures only)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.configs_table:
        import paper_2510_17734_gb300 as bfc
        bfc.load()
        if rank == 0:
            print(json.dumps({"configs": run_config_table(bfc)}), flush=True)
        return 0
    if args.learned_only:
        import paper_2510_17734_gb300 as bfc
        bfc.load()
        if rank == 0:
            res = run_learned(bfc, n_train=args.learned_train, n_test=args.learned_test,
                              epochs=args.learned_epochs)
            print(json.dumps({"learned_start": res}), flush=True)
        return 0
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        return run_bfc(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
