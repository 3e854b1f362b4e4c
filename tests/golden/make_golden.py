"""Writes the stored inputs under tests/golden/ from ``synth`` and ``oracle`` only.

c4h6_seed1_relaxed.txt: the C4H6 (seed 1) geometry relaxed by 300 damped
oracle XL-BOMD steps (velocities scaled by 0.9 per step, T_e = 1000 K,
m = 4, dt = 0.5 fs, synthetic table seed 1).  The paper relaxes its
structures before MD (Results, "Methanol IR Spectrum"); the relaxed geometry
is the start of the energy-conservation runs.

Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import dynamics as dyn, hamiltonian as ham  # noqa: E402


def relaxed_c4h6():
    tab = synth.synthetic_table(1)
    mol = synth.c4h6(1)
    sysm = ham.System(mol.Z, tab)
    cfg = dyn.Config(Te=1000.0, dt=0.5, m=4)
    st = dyn.State(sysm, mol.R, np.zeros_like(mol.R), cfg)
    for _ in range(300):
        st.step()
        st.V *= 0.9
    return st.R


if __name__ == "__main__":
    R = relaxed_c4h6()
    np.savetxt(os.path.join(HERE, "c4h6_seed1_relaxed.txt"), R, fmt="%.15e",
               header="C4H6 seed 1 relaxed by damped oracle XL-BOMD (see make_golden.py); Angstrom")
