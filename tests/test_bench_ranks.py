"""The host logic of bench.py's multi-GPU mode, run as two gloo ranks on the
CPU: every rank updates its own factorization (distinct seeded workloads, no
data-path collective), the job's timed region is the slowest rank's, and the
reported value is the units of all ranks over that time."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 180.0][rank]
        slow = bench.slowest_rank_ms(local_ms, dist, "cpu")
        bench.M = bench.N = 64
        _, _, _, _, ups = bench.workload(rank, 2)
        out.put((rank, slow, bench.job_throughput(world, 10, slow), ups[0][0].copy()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_and_sum_the_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, s0, v0, b0), (_, s1, v1, b1) = res
    assert s0 == s1 == 180.0
    assert v0 == v1 == pytest.approx(2 * 10 / 0.18)
    assert not np.array_equal(b0, b1)  # independent replicas, distinct streams


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.slowest_rank_ms(42.5, None, "cpu") == 42.5
    assert bench.job_throughput(1, 10, 2000.0) == pytest.approx(5.0)
