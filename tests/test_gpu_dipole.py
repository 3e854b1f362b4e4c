"""GPU dipole moment (the per-step record's `dipole`, the observable behind the
paper's IR spectrum, Results) against the oracle, through the C ABI.

On a polar organic molecule (C/N/O/H), teacher-forced at a perturbed density
and after MD steps: the GPU's dipole equals the oracle's formula applied to
the GPU's own R and D0 to FP64 rounding (it is a linear function of D0), and
the oracle's dipole of its own evaluation within the D0 parity bar times the
molecule's size."""
import numpy as np
import pytest

import paper_2303_00689_gb300 as kx
import synth
from oracle import dynamics as dyn, hamiltonian as ham
from tests.gpu_helpers import create, oracle_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_00689_gb300 import build
    build.build()


def _polar(seed=11, natoms=9):
    rng = np.random.default_rng(seed)
    for _ in range(50):
        mol = synth.organic_molecule(rng, natoms)
        if any(int(z) in (7, 8) for z in mol.Z):
            return mol
    raise RuntimeError("no polar molecule drawn")


@pytest.mark.parametrize("prec", [kx.SIM_PREC_FP64, kx.SIM_PREC_MIXED])
def test_dipole_record_matches_oracle(prec):
    mol = _polar()
    sysm = oracle_system(mol)
    cfg = dyn.Config(Te=1000.0, dt=0.5, m=4)
    rng = np.random.default_rng(5)
    Y = rng.normal(size=(sysm.n, sysm.n)) * 1e-3
    X = dyn.initial_guess(sysm) + Y + Y.T
    ev = dyn.evaluate(sysm, mol.R, X, cfg, krylov=False)
    mu_oracle = ham.dipole(sysm, mol.R, ev["D"])
    h = create(mol, dict(Te=1000.0, dt=0.5, m_max=4, m_min=4, precision=prec), P0=X)
    try:
        rec = kx.sim_last_result(h)
        R, _, _, D = kx.sim_get_state(h, mol.natoms)
        mu = np.array(rec["dipole"])
        own = ham.dipole(sysm, R, D)
        scale = 1.0 + np.abs(own).max()
        assert np.max(np.abs(mu - own)) < 1e-12 * scale * mol.natoms
        tol = (1e-9 if prec == kx.SIM_PREC_FP64 else 1e-6) * 10 * mol.natoms
        assert np.max(np.abs(mu - mu_oracle)) < tol
        assert np.linalg.norm(mu_oracle) > 0.05
        # and after three MD steps, against the GPU's own state
        recs = kx.sim_step(h, 3)
        R, _, _, D = kx.sim_get_state(h, mol.natoms)
        own = ham.dipole(sysm, R, D)
        assert np.max(np.abs(np.array(recs[-1]["dipole"]) - own)) < 1e-12 * scale * mol.natoms
        assert len({tuple(r["dipole"]) for r in recs}) == 3        # it moves with the atoms
    finally:
        kx.sim_destroy(h)
