"""Shared set-up for the GPU parity tests: the same seeded inputs go to the
CUDA library (through the C ABI) and to the CPU oracle."""
import numpy as np

import paper_2303_00689_gb300 as kx
import synth
from oracle import dynamics as dyn, hamiltonian as ham

TABLE_SEED = 1


def table(seed=TABLE_SEED):
    return synth.synthetic_table(seed)


def create(mol, cfg_kw=None, V=None, P0=None, tab=None):
    tab = tab or table()
    cfg = kx.sim_config_default(**(cfg_kw or {}))
    h = kx.sim_create(cfg, kx.param_table(synth.table_to_array(tab)), mol.Z, mol.R, V=V,
                      charge=mol.charge, P0=P0)
    return h


def oracle_system(mol, tab=None):
    return ham.System(mol.Z, tab or table(), charge=mol.charge)


def max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))
