"""Host logic of bench.py's multi-GPU path (replicas, one process per GPU):
the step time is the max over ranks and the job's throughput sums the
replicas' work.  Run as two gloo processes on the CPU."""
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
