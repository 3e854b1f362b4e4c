"""Seeded Maxwell-Boltzmann initial velocities (Angstrom/fs), zero net momentum."""
import numpy as np

MASS = {1: 1.008, 6: 12.011, 7: 14.007, 8: 15.999}   # amu
_KB = 8.617333262e-5        # eV/K
_EV_PER_AMU = 9.648533212e-3  # (Angstrom/fs)^2 per (eV/amu)


def maxwell_boltzmann(Z, temperature=300.0, seed=0):
    rng = np.random.default_rng(np.random.SeedSequence([0x7E1, seed]))
    m = np.array([MASS[int(z)] for z in Z])
    sigma = np.sqrt(_KB * temperature * _EV_PER_AMU / m)
    v = rng.normal(size=(len(Z), 3)) * sigma[:, None]
    v -= (m[:, None] * v).sum(axis=0) / m.sum()
    return v
