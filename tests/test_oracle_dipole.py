"""Pins of the oracle's dipole moment (the observable behind the paper's IR
spectrum, Results; NDDO form read in oracle/hamiltonian.py).

* Hellmann-Feynman: with a uniform field E added to the Hamiltonian
  (h -> h + E . r on the on-site position operator, V_nn -> V_nn - E . sum Z' R),
  the SCF free energy Omega(E) satisfies dOmega/dE_k = -mu_k at E = 0.  The
  derivative is taken by central differences of converged SCF energies, so a
  wrong factor on the s-p term, a wrong sign or a density counted per spin
  instead of in total fails it.
* Origin: a neutral molecule's dipole does not depend on where the origin
  is; a cation's moves by its charge times the shift.
* Limits: with D1 = 0 (no s-p term) the dipole is the point-charge sum
  sum_A (Z'_A - N_A) R_A of the Mulliken-like populations N_A = 2 sum D_mu,mu.
"""
import numpy as np
import pytest

import synth
from oracle import hamiltonian as ham, electronic as el
from tests.gpu_helpers import table

TE = 1000.0


def _polar_molecule(seed=11, natoms=9):
    rng = np.random.default_rng(seed)
    for _ in range(50):
        mol = synth.organic_molecule(rng, natoms)
        if any(int(z) in (7, 8) for z in mol.Z):
            return mol
    raise RuntimeError("no polar molecule drawn")


def _scf(sysm, R, hfield=None, vshift=0.0, tol=1e-12, P0=None):
    pairs = ham.PairCache(sysm, R)
    h, Vnn = ham.core_hamiltonian(sysm, R, pairs)
    if hfield is not None:
        h = h + hfield
    P = np.eye(sysm.n) * (sysm.nocc / sysm.n) if P0 is None else P0.copy()
    for it in range(4000):
        G = ham.two_electron(sysm, R, P, pairs)
        D, eps, Q, f, mu = el.density(h + G, sysm.nocc, TE)
        err = np.abs(D - P).max()
        if err < tol:
            break
        P = 0.3 * P + 0.7 * D
    else:
        raise RuntimeError(f"SCF {err:.2e}")
    G = ham.two_electron(sysm, R, D, pairs)
    omega = ham.electronic_energy_terms(h, G, D, D) - 2.0 * TE * el.entropy(f) + Vnn + vshift
    return D, omega


@pytest.fixture(scope="module")
def polar():
    mol = _polar_molecule()
    sysm = ham.System(mol.Z, table(), charge=mol.charge)
    D, _ = _scf(sysm, mol.R)
    return mol, sysm, D


def test_dipole_is_minus_the_field_derivative_of_the_scf_energy(polar):
    mol, sysm, D0 = polar
    mu = ham.dipole(sysm, mol.R, D0)
    M = ham.dipole_operator(sysm, mol.R)
    nuc = (sysm.elem["zcore"][:, None] * mol.R).sum(axis=0)
    h_step = 1e-4                                  # V / Angstrom
    fd = np.zeros(3)
    for k in range(3):
        om = []
        for sgn in (1.0, -1.0):
            Ek = sgn * h_step
            _, o = _scf(sysm, mol.R, hfield=Ek * M[k], vshift=-Ek * nuc[k], P0=D0)
            om.append(o)
        fd[k] = -(om[0] - om[1]) / (2.0 * h_step)
    assert np.linalg.norm(mu) > 0.05              # a genuinely polar case
    assert np.max(np.abs(fd - mu)) < 1e-6 * max(1.0, np.abs(mu).max()), (fd, mu)


def test_neutral_dipole_is_origin_independent_and_ions_shift_by_their_charge(polar):
    mol, sysm, D = polar
    t = np.array([3.0, -1.5, 2.25])
    mu0 = ham.dipole(sysm, mol.R, D)
    mu1 = ham.dipole(sysm, mol.R + t, D)
    assert np.max(np.abs(mu1 - mu0)) < 1e-12
    # a dication of the same molecule (two electrons fewer; D rescaled is a valid per-spin density)
    ion = ham.System(mol.Z, table(), charge=2)
    Dion = D * (ion.nocc / sysm.nocc)
    q = 2.0 * (sysm.nocc - ion.nocc)
    assert q == 2.0
    d = ham.dipole(ion, mol.R + t, Dion) - ham.dipole(ion, mol.R, Dion)
    assert np.max(np.abs(d - q * t)) < 1e-12


def test_without_the_sp_term_the_dipole_is_the_point_charge_sum(polar):
    mol, sysm, D = polar
    sysm.elem["D1"] = np.zeros_like(sysm.elem["D1"])
    try:
        mu = ham.dipole(sysm, mol.R, D)
    finally:
        sysm.elem["D1"] = ham.System(mol.Z, table(), charge=mol.charge).elem["D1"]
    Db = sysm.pad(D)
    pops = np.array([2.0 * np.trace(Db[A, :, A, :]) for A in range(sysm.N)])
    q = sysm.elem["zcore"] - pops
    assert np.max(np.abs(mu - (q[:, None] * mol.R).sum(axis=0))) < 1e-12
