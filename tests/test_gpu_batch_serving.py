"""Molecule batches, CUDA-graph steps and the trajectory server, through the C ABI.

* A step replayed from a CUDA graph is the same kernel sequence on the same
  buffers: R, V, X and the step records are bitwise those of direct launches.
* sim_batch_step interleaves independent handles on their own streams: each
  molecule's trajectory is bitwise the one it has when stepped alone.
* The server (continuous batching under a memory budget) returns for every
  trajectory exactly what it returns when that trajectory runs alone, admits
  no more than the budget allows, reports per-trajectory errors without
  disturbing the others, and its trajectories match the oracle.
"""
import numpy as np
import pytest

import paper_2303_00689_gb300 as kx
import synth
from oracle import dynamics as dyn
from tests.gpu_helpers import create, oracle_system, max_abs, table

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_00689_gb300 import build
    build.build()


def _small_batch(k=4, seed=3):
    mols = synth.molecule_batch(seed=seed, count=32, nmin=12, nmax=40)
    return mols[:k]


def _cfg(**kw):
    base = dict(Te=1000.0, dt=0.5, m_max=4, m_min=4, scf_tol=1e-8, scf_krylov=1, scf_max=200, scf_accept=1)
    base.update(kw)
    return kx.sim_config_default(**base)


def _table():
    return kx.param_table(synth.table_to_array(table()))


def _state(h, N):
    R, V, F, _ = kx.sim_get_state(h, N)
    return R, V, F, kx.sim_get_matrix(h, kx.SIM_MAT_X)


@pytest.mark.parametrize("precision", [kx.SIM_PREC_FP64, kx.SIM_PREC_MIXED])
def test_graph_steps_are_bitwise_direct_steps(precision):
    mol = synth.c4h6(1)
    V = synth.maxwell_boltzmann(mol.Z, 300.0, seed=1)
    cfg = _cfg(precision=precision)
    ha = kx.sim_create(cfg, _table(), mol.Z, mol.R, V=V)
    hb = kx.sim_create(cfg, _table(), mol.Z, mol.R, V=V)
    try:
        kx.sim_enable_graphs(hb)
        ra = kx.sim_step(ha, 11)        # crosses the 8-slot ring more than once
        rb = kx.sim_step(hb, 11)
        assert ra == rb
        for a, b in zip(_state(ha, mol.natoms), _state(hb, mol.natoms)):
            assert np.array_equal(a, b)
        kx.sim_step_async(hb, 3)
        kx.sim_step_async(ha, 3)
        assert kx.sim_records(ha, 3) == kx.sim_records(hb, 3)
        kx.sim_enable_graphs(hb, False)
        assert kx.sim_step(ha, 2) == kx.sim_step(hb, 2)
    finally:
        kx.sim_destroy(ha)
        kx.sim_destroy(hb)


@pytest.mark.parametrize("graphs", [False, True])
def test_batch_step_equals_individual_steps(graphs):
    mols = _small_batch(4)
    cfg = _cfg(precision=kx.SIM_PREC_MIXED)
    Vs = [synth.maxwell_boltzmann(m.Z, 300.0, seed=10 + i) for i, m in enumerate(mols)]
    hs_b = [kx.sim_create(cfg, _table(), m.Z, m.R, V=v, charge=m.charge) for m, v in zip(mols, Vs)]
    hs_i = [kx.sim_create(cfg, _table(), m.Z, m.R, V=v, charge=m.charge) for m, v in zip(mols, Vs)]
    try:
        if graphs:
            for h in hs_b:
                kx.sim_enable_graphs(h)
        kx.sim_batch_step(hs_b, 6)
        for h in hs_i:
            kx.sim_step(h, 6)
        for m, hb, hi in zip(mols, hs_b, hs_i):
            assert kx.sim_records(hb, 6) == kx.sim_records(hi, 6)
            for a, b in zip(_state(hb, m.natoms), _state(hi, m.natoms)):
                assert np.array_equal(a, b)
    finally:
        for h in hs_b + hs_i:
            kx.sim_destroy(h)


def _run_server(requests, **server_kw):
    out = {}
    with kx.Server(**server_kw) as srv:
        tickets = {name: srv.submit(**req) for name, req in requests.items()}
        srv.drain(600.0)
        for name, t in tickets.items():
            out[name] = srv.poll(t)
        stats = srv.stats()
    return out, stats


def _requests():
    mols = _small_batch(3, seed=4)
    c4 = synth.c4h6(1)
    reqs = {"c4h6": dict(cfg=_cfg(precision=kx.SIM_PREC_MIXED), table=_table(), Z=c4.Z, R=c4.R,
                         V=synth.maxwell_boltzmann(c4.Z, 300.0, seed=1), nsteps=12)}
    for i, m in enumerate(mols):
        reqs[f"mol{i}"] = dict(cfg=_cfg(precision=kx.SIM_PREC_MIXED), table=_table(), Z=m.Z, R=m.R,
                               V=synth.maxwell_boltzmann(m.Z, 300.0, seed=20 + i), charge=m.charge,
                               nsteps=8 + 3 * i)
    return reqs


@pytest.mark.parametrize("graphs", [False, True])
def test_server_results_do_not_depend_on_the_mix(graphs):
    reqs = _requests()
    alone, _ = _run_server({"c4h6": reqs["c4h6"]}, use_graphs=graphs)
    mixed, stats = _run_server(reqs, use_graphs=graphs, max_active=8)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["max_active_seen"] >= 2
    a, b = alone["c4h6"], mixed["c4h6"]
    assert a["status"] == b["status"] == kx.SIM_OK
    assert a["steps_done"] == b["steps_done"] == 12
    assert a["records"] == b["records"]
    for k in ("R", "V", "F"):
        assert np.array_equal(a[k], b[k])
    # and equal to the same trajectory run through sim_create + sim_step
    c4 = reqs["c4h6"]
    h = kx.sim_create(c4["cfg"], c4["table"], c4["Z"], c4["R"], V=c4["V"])
    try:
        recs = kx.sim_step(h, 12)
        R, V, F, _ = kx.sim_get_state(h, len(c4["Z"]))
        assert recs == b["records"]
        assert np.array_equal(R, b["R"]) and np.array_equal(F, b["F"])
    finally:
        kx.sim_destroy(h)
    assert stats["atom_steps"] == sum(len(r["Z"]) * r["nsteps"] for r in reqs.values())
    assert stats["step_p50_ms"] > 0.0 and stats["step_p99_ms"] >= stats["step_p50_ms"]


def test_server_memory_budget_serialises_admission():
    reqs = _requests()
    two = {k: reqs[k] for k in ("mol0", "mol1")}
    need = [kx.sim_estimate_bytes(r["cfg"], r["Z"]) for r in two.values()]
    res, stats = _run_server(two, hbm_budget_bytes=max(need) + min(need) // 2)
    assert stats["max_active_seen"] == 1
    assert all(r["status"] == kx.SIM_OK for r in res.values())
    with kx.Server(hbm_budget_bytes=min(need) // 2) as srv:
        with pytest.raises(kx.SimError) as e:
            srv.submit(**two["mol0"])
        assert e.value.code == kx.SIM_EINVAL


def test_server_reports_errors_per_trajectory():
    reqs = _requests()
    bad = dict(reqs["c4h6"], charge=1)            # odd electron count: rejected by sim_create
    res, stats = _run_server({"bad": bad, "good": reqs["mol0"]})
    assert res["bad"]["status"] == kx.SIM_EINVAL and "electron" in res["bad"]["error"]
    assert res["good"]["status"] == kx.SIM_OK and res["good"]["steps_done"] == reqs["mol0"]["nsteps"]
    assert stats["failed"] == 1 and stats["completed"] == 1


def test_server_trajectory_matches_oracle():
    """A served FP64 trajectory against the oracle trajectory (C4H6, 6 steps)."""
    c4 = synth.c4h6(1)
    sysm = oracle_system(c4)
    cfg = dyn.Config(Te=1000.0, dt=0.5, m=4)
    Dmin, _ = dyn.scf(sysm, c4.R, cfg)
    V = synth.maxwell_boltzmann(c4.Z, 300.0, seed=1)
    st = dyn.State(sysm, c4.R, V, cfg, X0=Dmin)
    E = []
    for _ in range(6):
        st.step()
        E.append(st.total_energy())
    req = dict(cfg=_cfg(scf_tol=1e-10, scf_krylov=0, scf_max=5000), table=_table(), Z=c4.Z, R=c4.R, V=V,
               nsteps=6)
    res, _ = _run_server({"a": req})
    r = res["a"]
    assert r["status"] == kx.SIM_OK
    assert max_abs(r["R"], st.R) < 1e-8
    assert max_abs(r["F"], st.ev["forces"]) < 1e-4
    assert max_abs([x["E_tot"] for x in r["records"]], E) < 1e-7


def test_whole_batch_graph_with_several_groups_equals_individual_steps():
    """Three 600-atom carbon packings (n = 2400): each persistent eigensolver
    grid takes one block on each of the 152 SMs (at most two such blocks fit
    on an SM), so the three do not fit on the device at once and the batch
    graph runs them as at least two groups one after the other (fork/join
    across groups); results bitwise equal to stepping each alone."""
    mols = [synth.carbon_packing(seed=40 + i, natoms=600) for i in range(3)]
    cfg = _cfg(precision=kx.SIM_PREC_MIXED, Te=3000.0)
    Vs = [synth.maxwell_boltzmann(m.Z, 300.0, seed=60 + i) for i, m in enumerate(mols)]
    P0s = [0.5 * np.eye(4 * m.natoms) for m in mols]
    hs_b = [kx.sim_create(cfg, _table(), m.Z, m.R, V=v, P0=p) for m, v, p in zip(mols, Vs, P0s)]
    hs_i = [kx.sim_create(cfg, _table(), m.Z, m.R, V=v, P0=p) for m, v, p in zip(mols, Vs, P0s)]
    b = kx.sim_batch_create(hs_b)
    try:
        assert kx.sim_batch_groups(b) >= 2
        kx.sim_batch_run(b, 3)
        for h in hs_i:
            kx.sim_step(h, 3)
        for m, hb, hi in zip(mols, hs_b, hs_i):
            assert kx.sim_records(hb, 3) == kx.sim_records(hi, 3)
            for a, c in zip(_state(hb, m.natoms), _state(hi, m.natoms)):
                assert np.array_equal(a, c)
    finally:
        kx.sim_batch_destroy(b)
        for h in hs_b + hs_i:
            kx.sim_destroy(h)


def test_whole_batch_graph_equals_individual_steps():
    """One CUDA graph per batch step (every molecule a branch): records and
    states bitwise equal to stepping each molecule alone, across the X ring."""
    mols = _small_batch(4, seed=5)
    cfg = _cfg(precision=kx.SIM_PREC_MIXED)
    Vs = [synth.maxwell_boltzmann(m.Z, 300.0, seed=30 + i) for i, m in enumerate(mols)]
    hs_b = [kx.sim_create(cfg, _table(), m.Z, m.R, V=v, charge=m.charge) for m, v in zip(mols, Vs)]
    hs_i = [kx.sim_create(cfg, _table(), m.Z, m.R, V=v, charge=m.charge) for m, v in zip(mols, Vs)]
    b = kx.sim_batch_create(hs_b)
    try:
        kx.sim_batch_run(b, 6)
        kx.sim_batch_run(b, 5)                  # 11 steps: the ring wraps
        for h in hs_i:
            kx.sim_step(h, 6)
            kx.sim_step(h, 5)
        for m, hb, hi in zip(mols, hs_b, hs_i):
            assert kx.sim_records(hb, 5) == kx.sim_records(hi, 5)
            for a, c in zip(_state(hb, m.natoms), _state(hi, m.natoms)):
                assert np.array_equal(a, c)
        kx.sim_step(hs_b[0], 1)                 # a member stepped on its own leaves the batch's phase
        with pytest.raises(kx.SimError) as e:
            kx.sim_batch_run(b, 1)
        assert e.value.code == kx.SIM_EINVAL
    finally:
        kx.sim_batch_destroy(b)
        for h in hs_b + hs_i:
            kx.sim_destroy(h)
