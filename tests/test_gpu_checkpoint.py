"""Checkpoint and resume through the C ABI: a trajectory saved with sim_save
and continued from sim_load is bitwise the uninterrupted trajectory (same
state, same kernels), for the FP64 and mixed paths and the XL-BOMD mode."""
import numpy as np
import pytest

import paper_2303_00689_gb300 as kx
import synth
from tests.gpu_helpers import table

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_00689_gb300 import build
    build.build()


@pytest.mark.parametrize("mode", ["fp64", "mixed", "xl"])
def test_resume_is_bitwise(mode, tmp_path):
    mol = synth.c4h6(1)
    kw = dict(Te=1000.0, dt=0.5, m_max=4, m_min=4, scf_tol=1e-9, scf_krylov=1, scf_max=200, scf_accept=1)
    if mode == "mixed":
        kw["precision"] = kx.SIM_PREC_MIXED
    if mode == "xl":
        kw.update(kernel=kx.SIM_KERNEL_XL, xl_c=0.9)
    cfg = kx.sim_config_default(**kw)
    tab = kx.param_table(synth.table_to_array(table()))
    h = kx.sim_create(cfg, tab, mol.Z, mol.R, V=synth.maxwell_boltzmann(mol.Z, 300.0, seed=1))
    path = str(tmp_path / "c4h6.ckpt")
    try:
        kx.sim_step(h, 4)
        kx.sim_save(h, path)
        ra = kx.sim_step(h, 5)
        sa = kx.sim_get_state(h, mol.natoms)
        Xa = kx.sim_get_matrix(h, kx.SIM_MAT_X)
    finally:
        kx.sim_destroy(h)
    g = kx.sim_load(path)
    try:
        rb = kx.sim_step(g, 5)
        sb = kx.sim_get_state(g, mol.natoms)
        assert ra == rb
        for a, b in zip(sa, sb):
            assert np.array_equal(a, b)
        assert np.array_equal(Xa, kx.sim_get_matrix(g, kx.SIM_MAT_X))
    finally:
        kx.sim_destroy(g)
