"""Host logic of bench.py.  The multi-GPU path (replicas, one process per
GPU): the step time is the max over ranks and the job's throughput sums the
replicas' work, run as two gloo processes on the CPU.  The per-kernel
roofline rows: algorithmic work over the measured kernel time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank          # rank 1 is the slower one
        m = bench.max_over_ranks(ms, dist, "cpu")
        out[rank] = (m, bench.job_throughput(1000, world, m))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        m, v = res[rank]
        assert m == 15.0                      # every rank sees the slowest rank's time
        assert v == pytest.approx(2 * 1000 / 15e-3)


def test_single_process_passes_through():
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_throughput(3774874, 1, 25.0) == pytest.approx(3774874 / 25e-3)


def test_kernel_rooflines_arithmetic():
    """Per-kernel roofline rows: algorithmic bytes or flops per launch over
    the mean CUDA-event time of that kernel, against the given peaks."""
    import synth
    p = synth.config(3)                     # n = 65536, L = 12, r = 8
    nnz, S = p.nnz, 1 << (p.L + 1)
    groups = bench.group_counts(p)
    grouped = {m: g for m, g in groups.items() if g < 0.1 * nnz}
    nplain = p.L - len(grouped)
    prof = {"env_right": (24, 24 * 0.1), "mid_gram": (2 * nplain, 2 * nplain * 1.0),
            "mid_gram_grp": (4 * len(grouped), 2 * len(grouped) * 0.5), "mid_solve": (24, 24 * 0.5),
            "eval": (2, 2 * 0.25)}
    stats = [{"refine_steps": p.L * S}, {"refine_steps": p.L * S}]
    rows = {r["kernel"]: r for r in bench.kernel_rooflines(p, prof, stats, {"hbm_gbs": 6000.0}, 80.0)}
    env = rows["k_env_right"]
    assert env["bytes"] == nnz * (16 * 8 + 4) + S * 64 * 8
    assert env["achieved"] == pytest.approx(env["bytes"] / 0.1e-3 / 1e9)
    assert env["frac"] == pytest.approx(env["achieved"] / 6000.0)
    assert env["ms_per_sweep"] == pytest.approx(1.2)
    args = type("A", (), {"n": 0})()
    gram = {r["kernel"]: r for r in bench.gram_rooflines(p, prof, 2, True, True, grouped,
                                                           {"bf16_tflops_sustained": 1700.0}, 80.0, 1.2, args)}
    # rows (2 m <= L + 1) or columns: level 1 has 16 rows per slice block
    assert groups[1] <= (1 << (p.L + 1)) * 16 and groups[p.L] <= (1 << (p.L + 1)) * 16
    tc = gram["k_mid_gram_tc"]
    assert tc["flop_per_launch"] == nnz * 8 * (64 * 65 // 2 + 64)
    assert tc["fp32_frac"] == pytest.approx(tc["flop_per_launch"] / 1e-3 / 1e12 / 80.0)
    assert tc["peak"] == pytest.approx(1700.0 * 1.1 / 2.25)
    grp = gram["k_group_sums + k_mid_gram_grp"]
    fl = (sum(grouped.values()) * 8 * (64 * 65 // 2 + 64) + len(grouped) * nnz * 8 * (64 + 8)) / len(grouped)
    assert grp["flop_per_launch"] == pytest.approx(fl)
    assert grp["frac"] == pytest.approx(fl / 0.5e-3 / 1e12 / 80.0)
    solve = rows["k_mid_solve"]
    assert solve["refine_steps_per_slice"] == pytest.approx(1.0)
    assert solve["bytes"] == S * (2080 + 64) * 8 + nnz * (16 * 8 + 4) + S * 64 * 24 + 4 * (S + 1)
    assert "k_eval" in rows and rows["k_eval"]["launch_ms"] == pytest.approx(0.25)


def test_reference_arm_json_line():
    """`bench.py --impl reference` times the oracle on the host cores and
    prints one JSON line with the arm's contract: the same metric and unit as
    the GPU arm, a cpu_baseline describing the run, and an e2e entry that
    moves no bytes between host and device."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                         cwd=root, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_traffic_constants_are_keyed_to_their_kernel_sources():
    """The measured DRAM traffic the bench reports belongs to a kernel's source
    as it was captured: the tensor-core Gram by its whole file, the solve by
    the span from warp_chol through k_mid_solve.  A change inside the span
    (simulated on a copy) changes the key, one outside it does not."""
    import hashlib
    for cap in (bench.TC_GRAM_TRAFFIC, bench.SOLVE_TRAFFIC):
        assert bench.kernel_source_sha(cap["source"], cap.get("span")) == cap["sha"]
    cap = bench.SOLVE_TRAFFIC
    with open(os.path.join(bench.ROOT, cap["source"])) as f:
        txt = f.read()
    a = txt.index(cap["span"][0]) + len(cap["span"][0])   # just past the start marker

    def key(t):
        return hashlib.sha256(t[t.index(cap["span"][0]):t.index(cap["span"][1])].encode()).hexdigest()[:16]

    assert key(txt) == cap["sha"]
    assert key(txt + "// outside\n") == cap["sha"]
    assert key(txt[:a] + "x" + txt[a:]) != cap["sha"]
