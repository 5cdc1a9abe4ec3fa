"""The bench's N-rank aggregation on CPU (gloo, world size 2): every rank gets the slowest rank's
step time and the whole job's rate (N replicas, weak scaling)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = [120.0, 180.0][rank]          # rank 1 is the slower one
        ms, value = bench.job_rate(elapsed, 3, 6.0e12, world, "cpu")
        out[rank] = (ms, value)
    finally:
        torch.distributed.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        ms, value = out[r]
        assert ms == pytest.approx(60.0)                     # 180 ms / 3 steps, on both ranks
        assert value == pytest.approx(2 * 6.0e12 / 0.060 / 1e9)


def test_one_rank_needs_no_process_group():
    import bench
    ms, value = bench.job_rate(100.0, 4, 1.0e12, 1)
    assert ms == 25.0
    assert value == pytest.approx(1.0e12 / 0.025 / 1e9)
