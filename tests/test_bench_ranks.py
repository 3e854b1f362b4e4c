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


def _replica_rank(rank, world, port, out):
    """A rank of the bench: steps its own C4H6 replica (the oracle on the CPU
    stands in for the GPU step) through bench.timed_replica."""
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import synth
    from oracle import dynamics as dyn, hamiltonian as ham
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mol = synth.c4h6(1)
        sysm = ham.System(mol.Z, synth.synthetic_table(1))
        V = synth.maxwell_boltzmann(mol.Z, 300.0, seed=10 + rank)      # a different replica per rank
        st = dyn.State(sysm, mol.R, V, dyn.Config(Te=1000.0, dt=0.5, m=4), X0=dyn.initial_guess(sysm))
        laps, total = bench.timed_replica(st.step, steps=3, warmup=1, barrier=dist.barrier,
                                          clock=bench.WallClock(), world=world, device="cpu")
        ms, value = bench.job_throughput(total, 3, mol.natoms, world)
        out.put((rank, st.t, len(laps), sum(laps), total, ms, value, float(st.total_energy())))
    finally:
        dist.destroy_process_group()


def test_two_replicas_step_through_the_bench_rank_logic():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    totals = {r[4] for r in res}
    assert len(totals) == 1                               # every rank reports the slowest rank's time
    total = totals.pop()
    for rank, t, nlaps, own, tot, ms, value in (r[:7] for r in res):
        assert t == 4 and nlaps == 3                      # 1 warm-up + 3 timed steps each
        assert own <= tot + 1e-9
        assert ms == pytest.approx(tot / 3)
        assert value == pytest.approx(2 * 10 / (ms / 1e3))
    assert res[0][7] != res[1][7]                         # two different replicas were stepped
