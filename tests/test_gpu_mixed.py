"""GPU parity of the mixed-precision path (tcgen05 BF16-split density and DMPT).

Tolerances: density matrix max-abs <= 1e-6; forces <= 1e-3 eV/A (the
reduced-precision bar).  The Krylov kernel result carries the ~2^-16 relative
error of the two-piece DMPT products.
"""
import numpy as np
import pytest

import paper_2303_00689_gb300 as kx
import synth
from oracle import dynamics as dyn
from tests.gpu_helpers import create, oracle_system, max_abs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_00689_gb300 import build
    build.build()


def _perturbed(D, seed, scale=1e-3):
    rng = np.random.default_rng(seed)
    Y = rng.normal(size=D.shape) * scale
    return D + Y + Y.T


def _organic(natoms, odd):
    """An organic molecule (C/N/O/H) with an odd or even number of orbitals."""
    rng = np.random.default_rng(np.random.SeedSequence([91, natoms]))
    for _ in range(200):
        mol = synth.organic_molecule(rng, natoms)
        n = int(sum(1 if z == 1 else 4 for z in mol.Z))
        if n % 2 == int(odd):
            return mol
    raise RuntimeError("no molecule of that parity drawn")


@pytest.mark.parametrize("kind", ["c4h6", "carbon100", "carbon200", "organic9-odd", "organic40-odd",
                                  "organic40-even", "organic120-odd"])
def test_mixed_evaluation_matches_oracle(kind):
    if kind == "c4h6":
        mol = synth.c4h6(1)
    elif kind.startswith("organic"):
        size, parity = kind[7:].split("-")
        mol = _organic(int(size), parity == "odd")
    else:
        mol = synth.carbon_packing(seed=7, natoms=int(kind[6:]))
    sysm = oracle_system(mol)
    cfg = dyn.Config(Te=3000.0, dt=0.5, m=4)
    X = _perturbed(dyn.initial_guess(sysm), 5)
    ev = dyn.evaluate(sysm, mol.R, X, cfg)
    h = create(mol, dict(Te=3000.0, dt=0.5, m_max=4, m_min=4, precision=kx.SIM_PREC_MIXED), P0=X)
    try:
        D = kx.sim_get_matrix(h, kx.SIM_MAT_D0)
        K = kx.sim_get_matrix(h, kx.SIM_MAT_KERNEL)
        _, _, F, _ = kx.sim_get_state(h, sysm.N)
        Q = kx.sim_get_matrix(h, kx.SIM_MAT_Q)
        Fk = kx.sim_get_matrix(h, kx.SIM_MAT_FOCK)
        eps = kx.sim_get_vector(h, 0)
        assert np.array_equal(D, D.T)
        assert max_abs(D, ev["D"]) < 1e-6
        assert max_abs(F, ev["forces"]) < 1e-3
        assert max_abs(K, ev["K"]) < 1e-3 * np.abs(ev["K"]).max()
        # eigenpairs of the mixed eigensolver (odd and even n: the tensor-core
        # back-transformation must have run, not only the tridiagonal vectors)
        assert np.abs(Fk @ Q - Q * eps).max() < 1e-6 * np.abs(Fk).max()
        assert np.abs(Q.T @ Q - np.eye(sysm.n)).max() < 1e-6
    finally:
        kx.sim_destroy(h)


def test_mixed_step_matches_oracle():
    mol = synth.carbon_packing(seed=7, natoms=100)
    sysm = oracle_system(mol)
    cfg = dyn.Config(Te=3000.0, dt=0.5, m=4)
    X = _perturbed(dyn.initial_guess(sysm), 6)
    V = synth.maxwell_boltzmann(mol.Z, 300.0, seed=2)
    st = dyn.State(sysm, mol.R, V, cfg, X0=X)
    st.step()
    h = create(mol, dict(Te=3000.0, dt=0.5, m_max=4, m_min=4, precision=kx.SIM_PREC_MIXED), V=V, P0=X)
    try:
        kx.sim_step(h, 1)
        R, Vg, F, D = kx.sim_get_state(h, sysm.N)
        Xg = kx.sim_get_matrix(h, kx.SIM_MAT_X)
        assert max_abs(Xg, st.X[0]) < 1e-6
        assert max_abs(D, st.ev["D"]) < 1e-6
        assert max_abs(F, st.ev["forces"]) < 1e-3
    finally:
        kx.sim_destroy(h)
