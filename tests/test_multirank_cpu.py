"""The N-GPU bench path on CPU: two gloo ranks run independent replicas, and
the job's time and throughput come from the slowest rank (the aggregation
bench.py uses under torchrun; no data-path collective exists)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, local_seconds, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.job_seconds(local_seconds[rank], world)
        out[rank] = (t, bench.job_throughput(1_000_000, 3, world, t))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    world = 2
    local = [0.5, 2.0]
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), local, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, v = res[r]
        assert t == pytest.approx(2.0)
        # 2 ranks x 3 replicas x 1e6 updates over 2 s
        assert v == pytest.approx(2 * 3 * 1e6 / 2.0 / 1e9)


def test_single_rank_needs_no_process_group():
    assert bench.job_seconds(1.25, 1) == 1.25
    assert bench.job_throughput(10**9, 2, 1, 4.0) == pytest.approx(0.5)
