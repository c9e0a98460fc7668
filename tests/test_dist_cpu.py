"""Replica aggregation of bench.py across ranks, with two gloo ranks on CPU:
the whole-job value counts every rank's keys over the slowest rank's time."""
from __future__ import annotations

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, ws: int, port: int, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    local_ms = [40.0, 50.0][rank]
    total, value = bench.aggregate_ranks(local_ms, keys_per_rank=1000, steps=10, ws=ws, device="cpu")
    q.put((rank, total, value))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, total, value in got:
        assert total == 50.0                       # max over ranks
        assert value == pytest.approx(2 * 1000 * 10 / 0.050)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    total, value = bench.aggregate_ranks(25.0, 100, 4, 1, "cpu")
    assert total == 25.0 and value == pytest.approx(100 * 4 / 0.025)
