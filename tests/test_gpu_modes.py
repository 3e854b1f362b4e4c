"""GPU parity of the kernel modes against the CPU oracle, through the C ABI.

* Original XL-BOMD kernel K = -c I (Results, Langevin run of C240 2+, c = 0.9
  there): one teacher-forced step, FP64 tolerances.
* Adaptive Krylov rank (eqs. 31-34 with the fit-error stop): the rank the GPU
  stops at equals the oracle's, K agrees, and the converged-rank result is
  bitwise the result of a fixed-rank run of that rank (the Krylov-loop kernels
  that run after convergence return without touching memory).
"""
import numpy as np
import pytest

import paper_2303_00689_gb300 as kx
import synth
from oracle import dynamics as dyn
from tests.gpu_helpers import create, oracle_system, max_abs

pytestmark = pytest.mark.gpu

D_TOL = 1e-6
F_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_00689_gb300 import build
    build.build()


def _perturbed(D, seed, scale=1e-3):
    rng = np.random.default_rng(seed)
    Y = rng.normal(size=D.shape) * scale
    return D + Y + Y.T


@pytest.mark.parametrize("c", [1.0, 0.9])
def test_xl_kernel_one_step_teacher_forced(c):
    mol = synth.c4h6(1)
    sysm = oracle_system(mol)
    cfg = dyn.Config(Te=1000.0, dt=0.5, xl_c=c)
    X = _perturbed(dyn.initial_guess(sysm), 5, scale=1e-2)
    V = synth.maxwell_boltzmann(mol.Z, 300.0, seed=1)
    st = dyn.State(sysm, mol.R, V, cfg, X0=X)
    K0 = st.ev["K"]
    st.step()
    h = create(mol, dict(Te=1000.0, dt=0.5, kernel=kx.SIM_KERNEL_XL, xl_c=c), V=V, P0=X)
    try:
        assert max_abs(kx.sim_get_matrix(h, kx.SIM_MAT_KERNEL), K0) < 1e-8 * np.abs(K0).max()
        recs = kx.sim_step(h, 1)
        R, Vg, F, D = kx.sim_get_state(h, sysm.N)
        assert max_abs(R, st.R) < 1e-12
        assert max_abs(Vg, st.V) < 1e-10
        assert max_abs(kx.sim_get_matrix(h, kx.SIM_MAT_X), st.X[0]) < 1e-10
        assert max_abs(D, st.ev["D"]) < D_TOL
        assert max_abs(F, st.ev["forces"]) < F_TOL
        K = kx.sim_get_matrix(h, kx.SIM_MAT_KERNEL)
        assert max_abs(K, st.ev["K"]) < 1e-8 * np.abs(st.ev["K"]).max()
        assert recs[0]["rank"] == 0
        assert abs(recs[0]["res_norm"] - np.linalg.norm(st.ev["D"] - st.X[0])) < 1e-9
    finally:
        kx.sim_destroy(h)


@pytest.fixture(scope="module")
def fragments():
    """40 C of chains and sheet fragments (no H, near-zero gap) at 5000 K."""
    mol = synth.carbon_fragments(seed=5, natoms=40)
    sysm = oracle_system(mol)
    X = _perturbed(dyn.initial_guess(sysm), 9)
    return mol, sysm, X


def test_adaptive_rank_matches_oracle(fragments):
    mol, sysm, X = fragments
    # oracle fit errors here: 0.896, 0.578, 0.539, 0.5388, 0.475, ... -> stop at rank 5
    tol, m_min, m_max = 0.5, 2, 8
    ev = dyn.evaluate(sysm, mol.R, X, dyn.Config(Te=5000.0, m=m_max, m_min=m_min, tol=tol))
    fits = ev["krylov"]["fit"]
    r = ev["krylov"]["rank"]
    assert 2 < r < m_max
    assert fits[r - 1] < 0.97 * tol and fits[r - 2] > 1.03 * tol   # the stop is not borderline
    h = create(mol, dict(Te=5000.0, dt=0.5, m_max=m_max, m_min=m_min, krylov_tol=tol), P0=X)
    try:
        rec = kx.sim_last_result(h)
        assert rec["rank"] == r
        assert abs(rec["fit_err"] - fits[r - 1]) < 1e-9
        K = kx.sim_get_matrix(h, kx.SIM_MAT_KERNEL)
        assert max_abs(K, ev["K"]) < 1e-7 * np.abs(ev["K"]).max()
        assert max_abs(kx.sim_get_matrix(h, kx.SIM_MAT_D0), ev["D"]) < D_TOL
    finally:
        kx.sim_destroy(h)


@pytest.mark.parametrize("precision", [kx.SIM_PREC_FP64, kx.SIM_PREC_MIXED])
def test_adaptive_rank_equals_fixed_rank_bitwise(fragments, precision):
    mol, sysm, X = fragments
    V = synth.maxwell_boltzmann(mol.Z, 300.0, seed=5)
    base = dict(Te=5000.0, dt=0.5, precision=precision)
    ha = create(mol, dict(base, m_max=8, m_min=2, krylov_tol=0.5), V=V, P0=X)
    try:
        r = kx.sim_last_result(ha)["rank"]
        hf = create(mol, dict(base, m_max=r, m_min=r), V=V, P0=X)
        try:
            assert np.array_equal(kx.sim_get_matrix(ha, kx.SIM_MAT_KERNEL),
                                  kx.sim_get_matrix(hf, kx.SIM_MAT_KERNEL))
            kx.sim_step(ha, 1)
            kx.sim_step(hf, 1)
            assert np.array_equal(kx.sim_get_matrix(ha, kx.SIM_MAT_X), kx.sim_get_matrix(hf, kx.SIM_MAT_X))
        finally:
            kx.sim_destroy(hf)
    finally:
        kx.sim_destroy(ha)


@pytest.mark.parametrize("m", [2, 4])
def test_krylov_scf_matches_oracle(m):
    """sim_create with scf_krylov: the low-rank Krylov SCF reaches the oracle's
    ground state (same fixed point; the iteration counts agree within one)."""
    mol = synth.c4h6(1)
    sysm = oracle_system(mol)
    cfg = dyn.Config(Te=1000.0, scf_tol=1e-10)
    D_ref, it_ref, _ = dyn.scf_krylov(sysm, mol.R, cfg, m=m)
    h = create(mol, dict(Te=1000.0, m_max=m, m_min=m, scf_tol=1e-10, scf_krylov=1))
    try:
        it, res = kx.sim_scf_info(h)
        assert res < 1e-10
        assert abs(it - it_ref) <= 1
        assert max_abs(kx.sim_get_matrix(h, kx.SIM_MAT_X), D_ref) < 1e-9
    finally:
        kx.sim_destroy(h)


def test_bomd_steps_match_oracle():
    """Born-Oppenheimer comparison mode (SCF from the previous density at every
    step): three FP64 steps of C4H6 against the oracle's BOMD steps."""
    mol = synth.c4h6(1)
    sysm = oracle_system(mol)
    V = synth.maxwell_boltzmann(mol.Z, 300.0, seed=1)
    cfg = dyn.Config(Te=1000.0, dt=0.5, scf_tol=1e-10, bomd=True)
    st = dyn.State(sysm, mol.R, V, cfg)
    E = []
    for _ in range(3):
        st.step()
        E.append(st.total_energy())
    h = create(mol, dict(Te=1000.0, dt=0.5, scf_tol=1e-10, kernel=kx.SIM_KERNEL_BOMD), V=V)
    try:
        recs = kx.sim_step(h, 3)
        R, Vg, F, D = kx.sim_get_state(h, sysm.N)
        assert max_abs(R, st.R) < 1e-10
        assert max_abs(Vg, st.V) < 1e-9
        assert max_abs(F, st.ev["forces"]) < F_TOL
        assert max_abs(D, st.ev["D"]) < D_TOL
        assert max_abs([r["E_tot"] for r in recs], E) < 1e-7
        assert all(r["rank"] == 0 and r["res_norm"] < 1e-8 for r in recs)
        with pytest.raises(kx.SimError):
            kx.sim_enable_graphs(h)
    finally:
        kx.sim_destroy(h)


def test_langevin_steps_match_oracle(tmp_path):
    """Langevin thermostat (OBABO with Philox4x32-10 normals, same counters on
    both sides): three FP64 steps of C4H6 against the oracle; graph replays and a
    checkpoint resume reproduce the direct trajectory bitwise (the step counter
    of the random stream lives on the device and in the checkpoint)."""
    mol = synth.c4h6(1)
    sysm = oracle_system(mol)
    cfg = dyn.Config(Te=1000.0, dt=0.5, m=4, langevin_T=300.0, gamma=0.1, seed=77)
    Dmin, _ = dyn.scf(sysm, mol.R, cfg)
    V = synth.maxwell_boltzmann(mol.Z, 300.0, seed=1)
    st = dyn.State(sysm, mol.R, V, cfg, X0=Dmin)
    for _ in range(3):
        st.step()
    kw = dict(Te=1000.0, dt=0.5, m_max=4, m_min=4, langevin_gamma=0.1, langevin_T=300.0, langevin_seed=77)
    ha = create(mol, kw, V=V, P0=Dmin)
    hb = create(mol, kw, V=V, P0=Dmin)
    path = str(tmp_path / "langevin.ckpt")
    try:
        kx.sim_enable_graphs(hb)
        kx.sim_step(ha, 2)
        kx.sim_save(ha, path)
        ra = kx.sim_step(ha, 1)
        rb = kx.sim_step(hb, 3)
        R, Vg, F, D = kx.sim_get_state(ha, sysm.N)
        assert max_abs(R, st.R) < 1e-10
        assert max_abs(Vg, st.V) < 1e-9
        assert max_abs(F, st.ev["forces"]) < F_TOL
        assert max_abs(kx.sim_get_matrix(ha, kx.SIM_MAT_X), st.X[0]) < 1e-9
        assert ra[0] == rb[2]
        for a, b in zip(kx.sim_get_state(ha, sysm.N), kx.sim_get_state(hb, sysm.N)):
            assert np.array_equal(a, b)
        hc = kx.sim_load(path)
        try:
            rc = kx.sim_step(hc, 1)
            assert rc == ra
            assert np.array_equal(kx.sim_get_state(hc, sysm.N)[1], Vg)
        finally:
            kx.sim_destroy(hc)
    finally:
        kx.sim_destroy(ha)
        kx.sim_destroy(hb)
