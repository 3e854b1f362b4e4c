"""Pins of the oracle's Fock build, energy and forces (eqs. 3, 6, 13, 17, 22, 37)."""
import numpy as np
import pytest

import synth
from oracle import hamiltonian as ham, electronic as el, dynamics as dyn

TAB = synth.synthetic_table(1)
MOL = synth.c4h6(1)


def _full_eri(sysm, R):
    """Full n^4 ERI tensor assembled from one-centre and pair blocks (NDDO)."""
    N = sysm.N
    E = np.zeros((N, 4, N, 4, N, 4, N, 4))
    for A in range(N):
        E[A, :, A, :, A, :, A, :] = sysm.onec[A]
    for sel, W, _, _ in ham.PairCache(sysm, R).values():
        for p, (A, B) in enumerate(zip(sysm.pA[sel], sysm.pB[sel])):
            E[A, :, A, :, B, :, B, :] = W[p]
            E[B, :, B, :, A, :, A, :] = np.transpose(W[p], (2, 3, 0, 1))
    E = E.reshape(4 * N, 4 * N, 4 * N, 4 * N)
    o = sysm.orb
    return E[np.ix_(o, o, o, o)]


def test_fock_equals_textbook_closed_shell_form():
    """Per-spin eq. 3 equals h + sum P_t[(mu nu|lam sig) - (mu lam|nu sig)/2], P_t = 2P."""
    sysm = ham.System(MOL.Z, TAB)
    rng = np.random.default_rng(1)
    P = rng.normal(size=(sysm.n, sysm.n)) * 0.2
    P = P + P.T
    F, h, G, _ = ham.fock(sysm, MOL.R, P)
    eri = _full_eri(sysm, MOL.R)
    Pt = 2.0 * P
    G_ref = np.einsum("mnls,ls->mn", eri, Pt) - 0.5 * np.einsum("mlns,ls->mn", eri, Pt)
    assert np.abs(G - G_ref).max() < 1e-11
    assert np.abs(F - F.T).max() < 1e-12


def test_zero_two_electron_parameters_give_core_hamiltonian():
    tab0 = synth.synthetic_table(1, two_electron=False)
    sysm = ham.System(MOL.Z, tab0)
    P = np.eye(sysm.n) * 0.5
    F, h, G, _ = ham.fock(sysm, MOL.R, P)
    assert np.abs(G).max() == 0.0
    assert np.array_equal(F, h)


def _shadow_energy(sysm, R, X, Te, entropy_factor=2.0):
    F, h, G, Vnn = ham.fock(sysm, R, X)
    D, eps, Q, f, mu = el.density(F, sysm.nocc, Te)
    return ham.electronic_energy_terms(h, G, D, X) - entropy_factor * Te * el.entropy(f) + Vnn


def _fd_force(sysm, R, X, Te, A, k, h=1e-3, entropy_factor=2.0):
    vals = []
    for s in (-2, -1, 1, 2):
        Rp = R.copy()
        Rp[A, k] += s * h
        vals.append(_shadow_energy(sysm, Rp, X, Te, entropy_factor))
    return -(vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)


@pytest.mark.parametrize("Te", [1000.0, 20000.0])
def test_forces_match_finite_differences_of_shadow_energy(Te):
    """Eq. 22: at fixed X the D0 variation drops out, so F = -dU/dR exactly."""
    sysm = ham.System(MOL.Z, TAB)
    cfg = dyn.Config(Te=Te)
    D, _ = dyn.scf(sysm, MOL.R, cfg)
    rng = np.random.default_rng(0)
    Y = rng.normal(size=D.shape) * 1e-2
    X = D + Y + Y.T                       # away from self-consistency
    ev = dyn.evaluate(sysm, MOL.R, X, cfg, krylov=False)
    for A in (0, 5):
        for k in range(3):
            assert abs(_fd_force(sysm, MOL.R, X, Te, A, k) - ev["forces"][A, k]) < 1e-6


def test_entropy_factor_one_breaks_force_consistency():
    """Planted mistake: -T_e S (as printed in eq. 13) instead of -2 T_e S.

    With the wrong factor D0 is no longer the stationary point of eq. 12, so
    finite differences of U disagree with the eq. 37 forces at high T_e.
    """
    Te = 20000.0
    sysm = ham.System(MOL.Z, TAB)
    cfg = dyn.Config(Te=Te)
    D, _ = dyn.scf(sysm, MOL.R, cfg)
    ev = dyn.evaluate(sysm, MOL.R, D, cfg, krylov=False)
    errs = [abs(_fd_force(sysm, MOL.R, D, Te, 0, k, entropy_factor=1.0) - ev["forces"][0, k])
            for k in range(3)]
    assert max(errs) > 1e-2


def test_forces_sum_to_zero_and_energy_translation_invariant():
    sysm = ham.System(MOL.Z, TAB)
    cfg = dyn.Config(Te=1000.0)
    D, _ = dyn.scf(sysm, MOL.R, cfg)
    ev = dyn.evaluate(sysm, MOL.R, D, cfg, krylov=False)
    assert np.abs(ev["forces"].sum(axis=0)).max() < 1e-10
    ev2 = dyn.evaluate(sysm, MOL.R + np.array([1.0, -2.0, 0.5]), D, cfg, krylov=False)
    assert ev2["U"] == pytest.approx(ev["U"], abs=1e-9)
