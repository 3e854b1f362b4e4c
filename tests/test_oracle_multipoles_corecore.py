"""Pins of the oracle's point-charge sets and of its core-core term.

The paper names the MNDO/AM1 Hamiltonians (Introduction) without printing
their integrals, so the oracle's model is pinned to mathematics it must obey:

* every orbital product on an atom is replaced by point charges whose monopole,
  dipole and traceless second moments must equal those of the Slater-orbital
  product they stand for; the moments of the real orbitals are computed here
  by radial and angular quadrature, independently of the multipole lengths
  D1, D2 the oracle derives;
* far from the atom the two-centre integrals must follow the multipole
  expansion of those moments (dipole ~ 1/R^2, quadrupole ~ 1/R^3);
* at bonding distances the molecular-frame integrals contracted with the bond
  direction must equal a direct sum over charges placed in 3-D space;
* the core-core term is pinned by reductions in which all but one of its
  pieces vanish (exponentials off, Gaussians off, Gaussians flattened to a
  constant, one Gaussian sampled at its centre), by its decay rate, its
  R -> infinity limit and its symmetry under exchange of the two atoms.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import synth
from oracle import nddo

TAB = synth.synthetic_table(1)
E2 = nddo.E2


# ---------------------------------------------------------------------------
# moments of the real Slater orbital products by quadrature
# ---------------------------------------------------------------------------
def _radial(n, zeta, r):
    return (2 * zeta) ** (n + 0.5) / math.sqrt(math.factorial(2 * n)) * r ** (n - 1) * math.exp(-zeta * r)


def _radial_moment(n, za, zb, power):
    """int R_a R_b r^(2 + power) dr in bohr^power (zeta in 1/bohr)."""
    return integrate.quad(lambda r: _radial(n, za, r) * _radial(n, zb, r) * r ** (2 + power), 0, 80,
                          epsabs=1e-13, epsrel=1e-12, limit=200)[0]


def _ylm(slot, th, ph):
    """Real s / p_x / p_y / p_z angular functions."""
    if slot == 0:
        return 1.0 / math.sqrt(4 * math.pi)
    c = math.sqrt(3.0 / (4 * math.pi))
    return c * (math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th))[slot - 1]


def _angular(a, b, f):
    """int Y_a Y_b f(unit vector) dOmega."""
    def g(ph, th):
        u = (math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th))
        return _ylm(a, th, ph) * _ylm(b, th, ph) * f(u) * math.sin(th)
    return integrate.dblquad(g, 0, math.pi, 0, 2 * math.pi, epsabs=1e-12, epsrel=1e-11)[0]


def _orbital_moments(rec, a, b):
    """Monopole, dipole (3) and second moments (3x3) of chi_a chi_b, Angstrom."""
    n = int(rec["nprin"])
    za = rec["zeta_s"] if a == 0 else rec["zeta_p"]
    zb = rec["zeta_s"] if b == 0 else rec["zeta_p"]
    B = nddo.BOHR
    m0 = _radial_moment(n, za, zb, 0) * _angular(a, b, lambda u: 1.0)
    r1 = _radial_moment(n, za, zb, 1) * B
    r2 = _radial_moment(n, za, zb, 2) * B * B
    dip = np.array([r1 * _angular(a, b, lambda u, k=k: u[k]) for k in range(3)])
    sec = np.array([[r2 * _angular(a, b, lambda u, k=k, l=l: u[k] * u[l]) for l in range(3)] for k in range(3)])
    return m0, dip, sec


def _charge_moments(charges):
    m0 = sum(q for q, _, _ in charges)
    dip = sum(q * np.array(p, dtype=float) for q, p, _ in charges)
    sec = sum(q * np.outer(p, p) for q, p, _ in charges)
    return m0, dip, sec


def _traceless(sec):
    return sec - np.trace(sec) / 3.0 * np.eye(3)


@pytest.mark.parametrize("Z", [6, 7, 8])
def test_point_charge_sets_reproduce_orbital_product_moments(Z):
    """Monopole, dipole and traceless quadrupole of every sp product."""
    rec = TAB[Z]
    der = nddo.element_derived(rec)
    for prod, (a, b) in enumerate(nddo.PRODUCTS):
        ch = nddo._charges(prod, der["D1"], der["D2"], der["rho0"], der["rho1"], der["rho2"])
        m0, dip, sec = _charge_moments(ch)
        t0, tdip, tsec = _orbital_moments(rec, a, b)
        assert m0 == pytest.approx(t0, abs=1e-9), (prod, "monopole")
        assert np.abs(dip - tdip).max() < 1e-8, (prod, "dipole", dip, tdip)
        # the point-charge model carries multipoles up to the quadrupole; the
        # trace of the second moment (a spherical shell) is not represented
        assert np.abs(_traceless(sec) - _traceless(tsec)).max() < 1e-8, (prod, "quadrupole")


def test_hydrogen_s_is_a_single_monopole():
    der = nddo.element_derived(TAB[1])
    ch = nddo._charges(0, der["D1"], der["D2"], der["rho0"], der["rho1"], der["rho2"])
    assert len(ch) == 1 and ch[0][0] == 1.0 and ch[0][2] == der["rho0"]


# ---------------------------------------------------------------------------
# two-centre integrals: far field and a direct 3-D sum at bonding distances
# ---------------------------------------------------------------------------
def _pair_arrays(ZA, ZB):
    ea, eb = {}, {}
    for e, Z in ((ea, ZA), (eb, ZB)):
        r = dict(TAB[Z])
        r.update(nddo.element_derived(TAB[Z]))
        for k, v in r.items():
            e[k] = np.array([v], dtype=np.float64)
    return ea, eb


def _local(ZA, ZB, R):
    ea, eb = _pair_arrays(ZA, ZB)
    return nddo.local_to_tensor(nddo.local_eri(np.array([R]), ea, eb))[0]


def test_far_field_dipole_and_quadrupole():
    """(s p_sigma|ss) -> e^2 D/R^2 and (p_sig p_sig|ss) - (p_pi p_pi|ss) ->
    e^2 (Q_zz - Q_xx)/R^3 with D, Q from quadrature of the C orbitals."""
    rec = TAB[6]
    _, tdip, _ = _orbital_moments(rec, 0, 3)
    _, _, sec_zz = _orbital_moments(rec, 3, 3)
    _, _, sec_xx = _orbital_moments(rec, 1, 1)
    # expansion of q / |R z - r| to second order: q [1/R + z/R^2 + (3 z^2 - r^2)/(2 R^3)];
    # p_z p_z and p_x p_x have the same trace <r^2>, so their difference seen
    # along z is 3/2 (<p_z|z^2|p_z> - <p_x|z^2|p_x>) / R^3
    quad = 1.5 * (sec_zz[2, 2] - sec_xx[2, 2])
    for R in (300.0, 600.0):
        W = _local(6, 1, R)                 # B = hydrogen: a pure monopole
        # B sits at +R z': the +1/2 charge of s p_z at +D1 z' is closer to it
        assert W[0, 3, 0, 0] * R * R / E2 == pytest.approx(tdip[2], rel=2e-4)
        diff = (W[3, 3, 0, 0] - W[1, 1, 0, 0]) * R ** 3 / E2
        assert diff == pytest.approx(quad, rel=2e-4)


def _charge_cloud(kind, e, D1, D2, r0, r1, r2, pos):
    """Point charges (q, xyz, rho) of an orbital product in 3-D space.

    kind 'ss' | 'se' (s and the p orbital along unit vector e) | 'ee' (p_e p_e);
    the MNDO model: dipole +-1/2 at +-D1 e; linear quadrupole +1/4 at +-2 D2 e
    and -1/2 at the nucleus on top of the unit monopole."""
    e = np.asarray(e, dtype=float)
    pos = np.asarray(pos, dtype=float)
    if kind == "ss":
        return [(1.0, pos, r0)]
    if kind == "se":
        return [(0.5, pos + D1 * e, r1), (-0.5, pos - D1 * e, r1)]
    return [(1.0, pos, r0), (0.25, pos + 2 * D2 * e, r2), (0.25, pos - 2 * D2 * e, r2), (-0.5, pos, r2)]


def _cloud_energy(ca, cb):
    tot = 0.0
    for qa, pa, ra in ca:
        for qb, pb, rb in cb:
            d = pa - pb
            tot += qa * qb / math.sqrt(d @ d + (ra + rb) ** 2)
    return E2 * tot


@pytest.mark.parametrize("R", [1.25, 1.6, 2.4])
def test_bonding_distance_integrals_equal_a_direct_charge_sum(R):
    """Rotated (pair vector off-axis) molecular-frame integrals, contracted
    with the bond direction u or a perpendicular unit vector t, equal the
    direct sum over charges placed along u and t (C on A, O on B)."""
    ea, eb = _pair_arrays(6, 8)
    u = np.array([0.3, -0.5, 0.8])
    u /= np.linalg.norm(u)
    t = np.cross(u, [1.0, 0.0, 0.0])
    t /= np.linalg.norm(t)
    d = (R * u)[None, :]
    W, _, _ = nddo.pair_values(d, ea, eb)
    W = W[0]
    pa = lambda k: {kk: float(ea[kk][0]) for kk in ("D1", "D2", "rho0", "rho1", "rho2")}[k]
    pb = lambda k: {kk: float(eb[kk][0]) for kk in ("D1", "D2", "rho0", "rho1", "rho2")}[k]
    A0, B0 = np.zeros(3), R * u

    def cloud(kind, e, p, pos):
        return _charge_cloud(kind, e, p("D1"), p("D2"), p("rho0"), p("rho1"), p("rho2"), pos)

    def contract(va, vb, wa, wb):
        """sum over p slots: W[mu nu | lam sig] with p parts given by vectors"""
        def sl(v):
            return np.concatenate([[1.0], np.zeros(3)]) if v is None else np.concatenate([[0.0], v])
        return np.einsum("a,b,c,d,abcd->", sl(va), sl(vb), sl(wa), sl(wb), W)

    cases = [
        (("ss", None), ("ss", None), contract(None, None, None, None)),
        (("ee", u), ("ss", None), contract(u, u, None, None)),
        (("ee", t), ("ss", None), contract(t, t, None, None)),
        (("se", u), ("se", u), contract(None, u, None, u)),
        (("se", t), ("se", t), contract(None, t, None, t)),
        (("ee", u), ("ee", u), contract(u, u, u, u)),
        (("ee", t), ("ee", u), contract(t, t, u, u)),
        (("ee", t), ("ee", t), contract(t, t, t, t)),
    ]
    for (ka, va), (kb, vb), got in cases:
        ref = _cloud_energy(cloud(ka, va, pa, A0), cloud(kb, vb, pb, B0))
        assert got == pytest.approx(ref, rel=1e-12, abs=1e-12), (ka, kb)


# ---------------------------------------------------------------------------
# core-core term
# ---------------------------------------------------------------------------
def _enn(ZA, ZB, R, **over):
    ea, eb = _pair_arrays(ZA, ZB)
    for key, val in over.items():
        side, name = key.split("_", 1)
        (ea if side == "A" else eb)[name] = np.array([val], dtype=np.float64)
    d = np.array([[0.0, 0.0, R]])
    return float(nddo.pair_values(d, ea, eb)[2][0]), ea, eb


def _no_gauss():
    over = {}
    for s in ("A", "B"):
        for k in range(2):
            over[f"{s}_gauss_a{k}"] = 0.0
    return over


def _gss(ZA, ZB, R):
    return float(_local(ZA, ZB, R)[0, 0, 0, 0])


@pytest.mark.parametrize("R", [0.9, 1.5, 3.0])
def test_core_core_reduces_to_core_charges_times_ss_integral(R):
    """Exponentials off (alpha -> infinity) and no Gaussians: Z'_A Z'_B (ss|ss);
    alpha = 0 (both exponentials equal 1): three times that."""
    zz = TAB[6]["zcore"] * TAB[8]["zcore"]
    gss = _gss(6, 8, R)
    big = dict(_no_gauss(), A_alpha=1e6, B_alpha=1e6)
    assert _enn(6, 8, R, **big)[0] == pytest.approx(zz * gss, rel=1e-14)
    zero = dict(_no_gauss(), A_alpha=0.0, B_alpha=0.0)
    assert _enn(6, 8, R, **zero)[0] == pytest.approx(3.0 * zz * gss, rel=1e-14)
    one = dict(_no_gauss(), A_alpha=0.0, B_alpha=1e6)     # one exponential on, one off
    assert _enn(6, 8, R, **one)[0] == pytest.approx(2.0 * zz * gss, rel=1e-14)


def test_core_core_exponential_decays_at_each_atoms_own_rate():
    zz = TAB[6]["zcore"] * TAB[8]["zcore"]
    for side, other in (("A", "B"), ("B", "A")):
        alpha = TAB[6]["alpha"] if side == "A" else TAB[8]["alpha"]
        logs = []
        Rs = (1.2, 1.8)
        for R in Rs:
            e, _, _ = _enn(6, 8, R, **dict(_no_gauss(), **{f"{other}_alpha": 1e6}))
            logs.append(math.log(e / (zz * _gss(6, 8, R)) - 1.0))
        assert (logs[1] - logs[0]) / (Rs[1] - Rs[0]) == pytest.approx(-alpha, rel=1e-10)


def test_core_core_gaussians_of_both_atoms_enter_with_one_over_R():
    """Gaussians flattened (b = 0) to their amplitudes: Z'Z'/R sum of all four
    a_k; and a single narrow Gaussian sampled at its own centre gives a_k Z'Z'/R."""
    zz = TAB[6]["zcore"] * TAB[8]["zcore"]
    R = 1.7
    flat = {"A_alpha": 1e6, "B_alpha": 1e6}
    for s in ("A", "B"):
        for k in range(2):
            flat[f"{s}_gauss_b{k}"] = 0.0
    e, ea, eb = _enn(6, 8, R, **flat)
    asum = sum(float(x[f"gauss_a{k}"][0]) for x in (ea, eb) for k in range(2))
    assert e - zz * _gss(6, 8, R) == pytest.approx(zz * asum / R, rel=1e-12)
    for s, Z in (("A", 6), ("B", 8)):
        for k in range(2):
            c = TAB[Z][f"gauss_c{k}"]
            over = dict(_no_gauss(), A_alpha=1e6, B_alpha=1e6)
            over[f"{s}_gauss_a{k}"] = 0.3
            over[f"{s}_gauss_b{k}"] = 50.0
            e, _, _ = _enn(6, 8, c, **over)
            assert e - zz * _gss(6, 8, c) == pytest.approx(zz * 0.3 / c, rel=1e-12)
            # and it is a Gaussian in R - c: symmetric about the centre
            ep, _, _ = _enn(6, 8, c + 0.07, **over)
            em, _, _ = _enn(6, 8, c - 0.07, **over)
            gp = (ep - zz * _gss(6, 8, c + 0.07)) * (c + 0.07) / zz
            gm = (em - zz * _gss(6, 8, c - 0.07)) * (c - 0.07) / zz
            assert gp == pytest.approx(gm, rel=1e-10)
            assert gp == pytest.approx(0.3 * math.exp(-50.0 * 0.07 ** 2), rel=1e-10)


def test_core_core_is_symmetric_in_the_two_atoms():
    for R in (1.1, 1.6, 2.5):
        eAB, _, _ = _enn(6, 8, R)
        ea, eb = _pair_arrays(8, 6)
        eBA = float(nddo.pair_values(np.array([[0.0, 0.0, -R]]), ea, eb)[2][0])
        assert eAB == pytest.approx(eBA, rel=1e-14)


def test_core_core_far_limit_is_point_charge_repulsion():
    zz = TAB[6]["zcore"] * TAB[8]["zcore"]
    R = 400.0    # additive terms shift 1/R by (rho_A + rho_B)^2 / (2 R^2) ~ 1e-5 here
    e, _, _ = _enn(6, 8, R)
    assert e * R / (zz * E2) == pytest.approx(1.0, rel=3e-5)
