"""bench.py's multi-rank aggregation on CPU: two gloo ranks, each timing its own
replica, report the job throughput from the slowest rank (replicas only: no
data-path collective, the one all-reduce is the timing maximum)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        my_ms = 1000.0 + 500.0 * rank          # rank 1 is the slow one
        total = bench.max_over_ranks(my_ms, world, "cpu")
        ms, value = bench.job_throughput(total, steps=10, natoms_per_rank=840, world=world)
        out.put((rank, total, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_uses_the_slowest_rank():
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
    for rank, total, ms, value in res:
        assert total == 1500.0
        assert ms == pytest.approx(150.0)
        assert value == pytest.approx(2 * 840 / 0.150)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    ms, v = bench.job_throughput(2720.0, 10, 840, 1)
    assert ms == 272.0 and v == pytest.approx(840 / 0.272)
