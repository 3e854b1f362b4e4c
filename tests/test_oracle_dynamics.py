"""Pins of the oracle's integrator (eqs. 27-30, 35) and constant of motion (eq. 26)."""
import os

import numpy as np
import pytest

import synth
from oracle import hamiltonian as ham, dynamics as dyn

TAB = synth.synthetic_table(1)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_damping_coefficients_cancel_on_linear_trajectories():
    """sum c_k = 0 and sum k c_k = 0: the damping term of eq. 29 vanishes for X(t) linear in t."""
    k = np.arange(dyn.KMAX + 1)
    assert dyn.CK.sum() == 0.0
    assert (k * dyn.CK).sum() == 0.0
    assert len(dyn.CK) == dyn.KMAX + 1 == 7


def test_damped_recursion_is_stable_for_minus_identity_kernel():
    """With K = -I, e(t+dt) = (2 - kappa) e(t) - e(t-dt) + alpha sum c_k e(t-k dt) is a contraction."""
    a, c = dyn.ALPHA, dyn.CK
    coef = np.zeros(dyn.KMAX + 2)
    coef[0] = 1.0
    coef[1] = -(2.0 - dyn.KAPPA) - a * c[0]
    coef[2] = 1.0 - a * c[1]
    for j in range(2, dyn.KMAX + 1):
        coef[j + 1] = -a * c[j]
    roots = np.roots(coef)
    assert np.abs(roots).max() < 0.96
    # without damping the recursion is only marginally stable
    assert np.abs(np.roots([1.0, -(2.0 - dyn.KAPPA), 1.0])).max() == pytest.approx(1.0, abs=1e-12)


def test_xl_kernel_equals_krylov_kernel_without_two_electron_terms():
    """G = 0 makes the residual Jacobian -I (eq. 31), so K = -I exactly: the
    Krylov kernel at rank 1 and 3 and the XL-BOMD kernel -c I with c = 1 agree,
    and c scales the XL kernel linearly."""
    mol = synth.c4h6(1)
    tab0 = synth.synthetic_table(1, two_electron=False)
    sysm = ham.System(mol.Z, tab0)
    rng = np.random.default_rng(3)
    X = dyn.initial_guess(sysm)
    A = rng.standard_normal(X.shape) * 1e-2
    X = X + 0.5 * (A + A.T)
    kx = dyn.evaluate(sysm, mol.R, X, dyn.Config(Te=1000.0, xl_c=1.0))["K"]
    for m in (1, 3):
        kk = dyn.evaluate(sysm, mol.R, X, dyn.Config(Te=1000.0, m=m))["K"]
        assert np.abs(kk - kx).max() < 1e-10 * np.abs(kx).max()
    k9 = dyn.evaluate(sysm, mol.R, X, dyn.Config(Te=1000.0, xl_c=0.9))["K"]
    assert np.abs(k9 - 0.9 * kx).max() < 1e-15 * np.abs(kx).max() + 1e-300
    # with the two-electron terms on, the exact kernel is no longer -I
    sysm1 = ham.System(mol.Z, TAB)
    kk = dyn.evaluate(sysm1, mol.R, X, dyn.Config(Te=1000.0, m=4))["K"]
    kx1 = dyn.evaluate(sysm1, mol.R, X, dyn.Config(Te=1000.0, xl_c=1.0))["K"]
    assert np.abs(kk - kx1).max() > 1e-3 * np.abs(kx1).max()


@pytest.mark.slow
def test_energy_conservation_and_dt_squared_scaling():
    """E_tot (eq. 26) fluctuates ~dt^2 and does not drift (Results, Gramicidin S NVE)."""
    mol = synth.c4h6(1)
    R0 = np.loadtxt(os.path.join(GOLDEN, "c4h6_seed1_relaxed.txt"))
    V0 = synth.maxwell_boltzmann(mol.Z, 300.0, seed=1)
    sysm = ham.System(mol.Z, TAB)
    stds, drifts = [], []
    for dt in (0.5, 0.25):
        cfg = dyn.Config(Te=1000.0, dt=dt, m=4)
        st = dyn.State(sysm, R0, V0, cfg)
        E = [st.total_energy()]
        for _ in range(int(60 / dt)):
            st.step()
            E.append(st.total_energy())
            X = st.X[0]
            assert np.array_equal(X, X.T)
        E = np.array(E)
        stds.append(E.std())
        drifts.append(dyn.energy_drift(np.arange(len(E)) * dt, E, sysm.N))
    assert 3.0 < stds[0] / stds[1] < 5.5
    # no systematic drift beyond the fluctuation over the 60 fs window
    for s, d in zip(stds, drifts):
        assert abs(d) * sysm.N * 0.060 < s
    assert stds[0] < 2e-3


def test_krylov_scf_reaches_the_linear_mixing_fixed_point():
    """The low-rank Krylov SCF (Results, "SCF Optimization") and linear mixing
    are different iterations with the same fixed point D[P] = P; the Krylov
    one needs far fewer iterations on a gapped molecule."""
    mol = synth.c4h6(1)
    sysm = ham.System(mol.Z, TAB)
    cfg = dyn.Config(Te=1000.0, scf_tol=1e-10)
    D_lin, it_lin = dyn.scf(sysm, mol.R, cfg)
    D_kry, it_kry, hist = dyn.scf_krylov(sysm, mol.R, cfg, m=3)
    assert np.abs(D_kry - D_lin).max() < 1e-9
    assert it_kry < it_lin / 2
    assert hist[-1] < 1e-10


def test_bomd_steps_conserve_the_born_oppenheimer_energy():
    """Born-Oppenheimer comparison mode: forces at the SCF ground state of each
    geometry.  E_kin + U is conserved to the Verlet error, which scales as dt^2
    (forces consistent with U_BO), and U at X = D_scf equals the ground-state
    energy evaluated from scratch at the final geometry."""
    mol = synth.c4h6(1)
    R0 = np.loadtxt(os.path.join(GOLDEN, "c4h6_seed1_relaxed.txt"))
    sysm = ham.System(mol.Z, TAB)
    V0 = synth.maxwell_boltzmann(mol.Z, 300.0, seed=1)
    stds = []
    for dt in (0.25, 0.125):
        cfg = dyn.Config(Te=1000.0, dt=dt, scf_tol=1e-11, bomd=True)
        st = dyn.State(sysm, R0, V0, cfg)
        E = [st.total_energy()]
        for _ in range(int(15.0 / dt)):
            st.step()
            E.append(st.total_energy())
        stds.append(np.std(E))
    assert 3.0 < stds[0] / stds[1] < 5.5
    D, _ = dyn.scf(sysm, st.R, dyn.Config(Te=1000.0, scf_tol=1e-11))
    fresh = dyn.evaluate(sysm, st.R, D, cfg, krylov=False)
    assert abs(fresh["U"] - st.ev["U"]) < 1e-8


def test_philox_known_answers():
    """Philox4x32-10 against the known-answer vectors published with the generator."""
    from oracle import rng
    cases = [((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
             ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
             ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
              (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1))]
    for ctr, key, want in cases:
        out = rng.philox4x32_10([[c] for c in ctr], key)
        assert tuple(int(o[0]) for o in out) == want


def test_langevin_half_steps_keep_the_maxwell_boltzmann_distribution():
    """The Ornstein-Uhlenbeck half step is exact for free particles: applied
    repeatedly it drives any velocities to <v^2> = k_B T ACC / M per component,
    and its normals are standard (mean 0, variance 1)."""
    from oracle import rng
    xi = rng.normals(200000, 0, 7, 12345)
    assert abs(xi.mean()) < 0.01 and abs(xi.var() - 1.0) < 0.01
    mol = synth.c4h6(1)
    sysm = ham.System(mol.Z, TAB)

    class Free(dyn.State):
        def __init__(self):
            self.sysm, self.cfg = sysm, dyn.Config(dt=0.5, langevin_T=500.0, gamma=0.5, seed=3)
            self.V = np.zeros((sysm.N, 3))
            self.t = 0

    st = Free()
    acc = np.zeros((sysm.N, 3))
    for t in range(4000):
        st.t = t
        st.thermostat(t % 2)
        if t >= 1000:
            acc += st.V ** 2
    v2 = acc / 3000
    # equipartition: sum M <v^2> / ACC = 3 N k_B T (about 1 % statistical error here)
    ratio = np.sum(sysm.mass[:, None] * v2) / dyn.ACC / (3 * sysm.N * dyn.KB * 500.0)
    assert abs(ratio - 1.0) < 0.05
