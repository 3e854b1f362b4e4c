"""Seeded synthetic NDDO parameter tables (raw parameters only).

The paper uses the AM1 Hamiltonian (Results section, first paragraph) and
cites MNDO/AM1/PM3 (Introduction); the parameter values themselves are not in
the paper.  The tables here are drawn uniformly inside ranges that fix the
physically meaningful signs and orderings only:

* U_ss < U_pp < 0 (one-centre one-electron energies, eV)
* beta_s, beta_p < 0 (resonance parameters, eV)
* G_ss, G_sp, G_pp, G_p2 > 0 and G_pp > G_p2 (so that H_pp > 0), H_sp > 0 (eV)
* Slater exponents zeta_s, zeta_p (1/bohr), core-core exponent alpha (1/Angstrom)
* two AM1-form Gaussian core-core terms per element (a in eV*Angstrom,
  b in 1/Angstrom^2, c in Angstrom)

Derived quantities (multipole lengths, additive terms, H_pp) are NOT computed
here; each consumer derives them from these raw values itself.
"""
import numpy as np

ELEMENTS = {1: "H", 6: "C", 7: "N", 8: "O"}

# Field order of one element record; the C header declares the same order.
FIELDS = (
    "Z", "norb", "nprin", "zcore", "mass",
    "U_ss", "U_pp", "zeta_s", "zeta_p", "beta_s", "beta_p",
    "G_ss", "G_sp", "G_pp", "G_p2", "H_sp", "alpha",
    "gauss_a0", "gauss_b0", "gauss_c0", "gauss_a1", "gauss_b1", "gauss_c1",
)

# (low, high) sampling ranges per element.  Orders of magnitude only.
_RANGES = {
    "H": dict(U_ss=(-13.0, -11.0), zeta_s=(1.10, 1.30), beta_s=(-7.0, -5.5),
              G_ss=(12.0, 14.0), alpha=(2.5, 3.0)),
    "C": dict(U_ss=(-53.0, -50.0), U_pp=(-40.5, -38.0), zeta_s=(1.75, 1.85),
              zeta_p=(1.65, 1.75), beta_s=(-16.0, -14.0), beta_p=(-9.0, -7.0),
              G_ss=(12.0, 13.0), G_sp=(11.2, 12.0), G_pp=(10.6, 11.4),
              G_p2=(9.5, 10.0), H_sp=(2.2, 2.6), alpha=(2.5, 2.7)),
    "N": dict(U_ss=(-72.0, -69.0), U_pp=(-58.0, -56.0), zeta_s=(2.0, 2.3),
              zeta_p=(2.0, 2.3), beta_s=(-21.0, -19.0), beta_p=(-19.0, -17.0),
              G_ss=(12.5, 13.5), G_sp=(12.0, 12.8), G_pp=(11.2, 12.0),
              G_p2=(10.2, 10.9), H_sp=(2.4, 2.9), alpha=(2.8, 3.0)),
    "O": dict(U_ss=(-98.0, -95.0), U_pp=(-79.0, -76.0), zeta_s=(2.6, 3.1),
              zeta_p=(2.5, 3.0), beta_s=(-30.0, -28.0), beta_p=(-30.0, -28.0),
              G_ss=(15.0, 15.8), G_sp=(14.2, 14.8), G_pp=(14.2, 14.8),
              G_p2=(12.6, 13.2), H_sp=(3.7, 4.1), alpha=(3.1, 3.3)),
}
_FIXED = {  # Z, orbitals, principal quantum number, core charge, mass (amu)
    "H": (1, 1, 1, 1.0, 1.008),
    "C": (6, 4, 2, 4.0, 12.011),
    "N": (7, 4, 2, 5.0, 14.007),
    "O": (8, 4, 2, 6.0, 15.999),
}


def synthetic_table(seed=1, two_electron=True):
    """Return {Z: {field: value}} for H, C, N, O drawn from ``seed``.

    ``two_electron=False`` zeroes every two-electron parameter (G's, H_sp);
    used by tests of the special case G == 0.
    """
    rng = np.random.default_rng(np.random.SeedSequence([0x5EED, seed]))
    table = {}
    for sym in ("H", "C", "N", "O"):
        Z, norb, nprin, zcore, mass = _FIXED[sym]
        rec = dict(Z=float(Z), norb=float(norb), nprin=float(nprin),
                   zcore=zcore, mass=mass)
        for key in FIELDS[5:17]:
            lo_hi = _RANGES[sym].get(key)
            rec[key] = float(rng.uniform(*lo_hi)) if lo_hi else 0.0
        for k in range(2):
            rec[f"gauss_a{k}"] = float(rng.uniform(0.05, 0.4))
            rec[f"gauss_b{k}"] = float(rng.uniform(4.0, 8.0))
            rec[f"gauss_c{k}"] = float(rng.uniform(1.2, 2.2))
        if not two_electron:
            for key in ("G_ss", "G_sp", "G_pp", "G_p2", "H_sp"):
                rec[key] = 0.0
        table[Z] = rec
    return table


def table_to_array(table):
    """Pack a table into a (4, len(FIELDS)) float64 array in H, C, N, O order."""
    return np.array([[table[Z][f] for f in FIELDS] for Z in (1, 6, 7, 8)],
                    dtype=np.float64)
