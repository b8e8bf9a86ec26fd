"""Multi-rank path of bench.py on CPU (gloo, world size 2).

CholeskyQR2 of one matrix does not shard here (each GPU factors its own
matrix: replicas), so the only cross-rank steps are host-side timing: a barrier
around the timed region and the maximum of the ranks' times. These run as two
gloo processes on the CPU.
"""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(ws)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env()[:2] == (ws, rank)
        bench.barrier(ws)
        ms_local = 10.0 + 5.0 * rank  # rank 1 is the slowest
        value, ms = bench.replica_throughput(ws, 1e12, ms_local)
        bench.barrier(ws)
        q.put((rank, value, ms))
    finally:
        dist.destroy_process_group()


def test_replica_timing_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, ms in got:
        assert ms == 15.0  # max over ranks
        assert value == pytest.approx(2 * 1e12 / 15e-3 / 1e12)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.allreduce_max(3.5, 1) == 3.5
    bench.barrier(1)
    value, ms = bench.replica_throughput(1, 2e12, 10.0)
    assert ms == 10.0 and value == pytest.approx(200.0)
