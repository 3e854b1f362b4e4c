"""Failure paths on the GPU in the forms that leave the device usable.

* NaN placed in the X history from the host (sim_set_state) reaches the
  forces and the Krylov kernel; the evaluation and the next step report
  SIM_ENUMERIC, and the handle recovers once a finite state is set again.
* The eigensolver's grid barrier is made to expire in a real step (wall-time
  limit 0 through the test hook): the kernel records the timeout and returns,
  the step reports SIM_ETIMEOUT, and after the limit is restored and the
  state re-established the handle steps bitwise like one that never failed.
* The tensor-core pipeline's bounded mbarrier wait, on a barrier nothing
  arrives at, expires and reports SIM_ETIMEOUT (no copy or tensor-core work
  is in flight in that test kernel).
* The server fails a trajectory whose atoms coincide (its integrals are not
  finite) and completes the others.
No test traps, faults or hangs the device: every wait involved is bounded and
NaN arithmetic only propagates.
"""
import numpy as np
import pytest

import paper_2303_00689_gb300 as kx
import synth
from tests.gpu_helpers import create

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_00689_gb300 import build
    build.build()


def _cfg(prec):
    return dict(Te=1000.0, dt=0.5, m_max=4, m_min=4, precision=prec, scf_tol=1e-8)


def _history(h):
    return np.stack([kx.sim_get_matrix(h, kx.SIM_MAT_XHIST + k) for k in range(7)])


@pytest.mark.parametrize("prec", [kx.SIM_PREC_FP64, kx.SIM_PREC_MIXED])
def test_nan_in_x_history_reports_enumeric_and_recovers(prec):
    mol = synth.c4h6(1)
    V = synth.maxwell_boltzmann(mol.Z, 300.0, seed=1)
    h = create(mol, _cfg(prec), V=V)
    try:
        kx.sim_step(h, 2, records=False)
        R, Vv, _, _ = kx.sim_get_state(h, mol.natoms)
        Xh = _history(h)
        bad = Xh.copy()
        bad[0, 3, 5] = bad[0, 5, 3] = np.nan
        with pytest.raises(kx.SimError) as e:
            kx.sim_set_state(h, Xhist=bad)
        assert e.value.code == kx.SIM_ENUMERIC
        with pytest.raises(kx.SimError) as e:
            kx.sim_step(h, 1, records=False)
        assert e.value.code == kx.SIM_ENUMERIC
        kx.sim_set_state(h, R=R, V=Vv, Xhist=Xh)       # finite state again
        rec = kx.sim_step(h, 2)
        assert all(np.isfinite(r["E_tot"]) for r in rec)
        assert np.all(np.isfinite(kx.sim_get_state(h, mol.natoms)[2]))
    finally:
        kx.sim_destroy(h)


@pytest.mark.parametrize("prec", [kx.SIM_PREC_FP64, kx.SIM_PREC_MIXED])
def test_expired_barrier_reports_etimeout_and_handle_recovers(prec):
    mol = synth.carbon_packing(seed=7, natoms=100)     # n = 400: a multi-block eigensolver grid
    V = synth.maxwell_boltzmann(mol.Z, 300.0, seed=3)
    P0 = 0.5 * np.eye(mol.norb)
    ha = create(mol, _cfg(prec), V=V, P0=P0)
    hb = create(mol, _cfg(prec), V=V, P0=P0)
    try:
        R, Vv, _, _ = kx.sim_get_state(ha, mol.natoms)
        Xh = _history(ha)
        kx.sim_debug_barrier_limit(0)
        try:
            with pytest.raises(kx.SimError) as e:
                kx.sim_step(ha, 1, records=False)
            assert e.value.code == kx.SIM_ETIMEOUT
        finally:
            kx.sim_debug_barrier_limit(2_000_000_000)
        kx.sim_set_state(ha, R=R, V=Vv, Xhist=Xh)
        ra = kx.sim_step(ha, 2)
        rb = kx.sim_step(hb, 2)
        assert ra == rb
        assert np.array_equal(kx.sim_get_state(ha, mol.natoms)[2], kx.sim_get_state(hb, mol.natoms)[2])
    finally:
        kx.sim_destroy(ha)
        kx.sim_destroy(hb)


def test_pipeline_mbarrier_wait_expires():
    assert kx.sim_debug_wait_expiry(4096) == kx.SIM_ETIMEOUT


def test_server_fails_the_trajectory_with_coincident_atoms_alone():
    tab = kx.param_table(synth.table_to_array(synth.synthetic_table(1)))
    cfg = kx.sim_config_default(Te=1000.0, dt=0.5, m_max=4, m_min=4, scf_tol=1e-8, scf_max=100)
    good = synth.c4h6(1)
    R_bad = good.R.copy()
    R_bad[1] = R_bad[0]                               # two carbons on one point
    with kx.Server(max_active=4) as srv:
        tb = srv.submit(cfg, tab, good.Z, R_bad, charge=good.charge, nsteps=3, records=False)
        tg = srv.submit(cfg, tab, good.Z, good.R, charge=good.charge, nsteps=3, records=False)
        srv.drain(120.0)
        rb, rg = srv.poll(tb), srv.poll(tg)
    assert rb["status"] in (kx.SIM_ENUMERIC, kx.SIM_ENOCONV)
    assert rg["status"] == kx.SIM_OK and rg["steps_done"] == 3
