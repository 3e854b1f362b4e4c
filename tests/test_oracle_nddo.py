"""Pins of the oracle's NDDO integrals against closed forms, quadrature and limits.

The paper prints no integral values (it cites MNDO/AM1/PM3, Introduction), so
these tests pin the oracle to mathematics it must satisfy rather than to
printed numbers.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import synth
from oracle import nddo, hamiltonian as ham

TAB = synth.synthetic_table(1)


def _pair(ZA, ZB, R, direction=(0.0, 0.0, 1.0)):
    rec = {ZA: TAB[ZA], ZB: TAB[ZB]}
    ea, eb = {}, {}
    for e, Z in ((ea, ZA), (eb, ZB)):
        r = dict(TAB[Z])
        r.update(nddo.element_derived(TAB[Z]))
        for k, v in r.items():
            e[k] = np.array([v], dtype=np.float64)
    d = np.array([direction], dtype=np.float64)
    d = d / np.linalg.norm(d) * R
    return d, ea, eb


def test_sto_1s1s_closed_form():
    # <1s|1s> = exp(-zR)(1 + zR + (zR)^2/3) for equal exponents (R in bohr)
    z = 1.2
    for Rb in (0.5, 1.4, 3.0):
        S = nddo.sto_overlap(np.array([Rb * nddo.BOHR]), 1, np.array([z]), "s", 1, np.array([z]), "s")[0]
        x = z * Rb
        assert S == pytest.approx(math.exp(-x) * (1 + x + x * x / 3), rel=1e-12)


def _sto_cart(n, zeta, kind, x, y, z):
    r = np.sqrt(x * x + y * y + z * z)
    N = (2 * zeta) ** (n + 0.5) / math.sqrt(math.factorial(2 * n))
    rad = N * r ** (n - 1) * np.exp(-zeta * r)
    if kind == "s":
        return rad / math.sqrt(4 * math.pi)
    ang = math.sqrt(3 / (4 * math.pi))
    if kind == "sig":
        return rad * ang * z / r
    return rad * ang * x / r


@pytest.mark.parametrize("nA,zA,kA,nB,zB,kB,Rb", [
    (2, 1.8, "s", 2, 1.7, "s", 2.6),
    (2, 1.8, "sig", 2, 1.7, "s", 2.6),
    (2, 1.7, "s", 2, 1.7, "sig", 2.4),
    (2, 1.7, "sig", 2, 2.1, "sig", 2.8),
    (2, 1.7, "pi", 2, 2.1, "pi", 2.8),
    (1, 1.2, "s", 2, 1.7, "sig", 2.0),
])
def test_sto_overlap_vs_quadrature(nA, zA, kA, nB, zB, kB, Rb):
    """Overlap in prolate spheroidal form vs brute-force quadrature in (rho, z)."""
    def integrand(rho, z):
        if kA == "pi":   # phi integral of cos^2 = pi; use x = rho on the phi = 0 plane
            a = _sto_cart(nA, zA, "pi", rho, 0.0, z)
            b = _sto_cart(nB, zB, "pi", rho, 0.0, z - Rb)
            return math.pi * rho * a * b
        a = _sto_cart(nA, zA, kA, rho, 0.0, z)
        b = _sto_cart(nB, zB, kB, rho, 0.0, z - Rb)
        return 2 * math.pi * rho * a * b
    val, _ = integrate.dblquad(lambda rho, z: integrand(rho, z), -25, 25 + Rb, 0, 25,
                               epsabs=1e-11, epsrel=1e-10)
    S = nddo.sto_overlap(np.array([Rb * nddo.BOHR]), nA, np.array([zA]), kA, nB, np.array([zB]), kB)[0]
    assert S == pytest.approx(val, abs=2e-8)


def test_multipole_lengths_match_their_definitions():
    """D1 = <ns|z|np_z> and D2^2 = <np|r^2|np>/5 by radial quadrature."""
    rec = TAB[6]
    der = nddo.element_derived(rec)
    n, zs, zp = 2, rec["zeta_s"], rec["zeta_p"]

    def R(zeta, r):
        return (2 * zeta) ** (n + 0.5) / math.sqrt(math.factorial(2 * n)) * r ** (n - 1) * math.exp(-zeta * r)
    rz = integrate.quad(lambda r: R(zs, r) * R(zp, r) * r ** 3, 0, 60)[0] / math.sqrt(3.0)
    r2 = integrate.quad(lambda r: R(zp, r) ** 2 * r ** 4, 0, 60)[0]
    assert der["D1"] == pytest.approx(rz * nddo.BOHR, rel=1e-9)
    assert der["D2"] == pytest.approx(math.sqrt(r2 / 5.0) * nddo.BOHR, rel=1e-9)


def test_one_center_limits():
    """R -> 0 on the same element reproduces G_ss, H_sp and H_pp."""
    d, ea, eb = _pair(6, 6, 1e-7)
    R, _ = nddo.local_frame(d)
    W = nddo.local_to_tensor(nddo.local_eri(R, ea, eb))[0]
    rec = TAB[6]
    assert W[0, 0, 0, 0] == pytest.approx(rec["G_ss"], rel=1e-9)
    assert W[0, 3, 0, 3] == pytest.approx(rec["H_sp"], rel=1e-6)
    assert W[1, 3, 1, 3] == pytest.approx(0.5 * (rec["G_pp"] - rec["G_p2"]), rel=1e-6)


def test_large_R_limit():
    """R -> infinity: monopole products give e^2/R, dipoles and quadrupoles vanish."""
    Rl = 2000.0
    d, ea, eb = _pair(6, 8, Rl)
    R, _ = nddo.local_frame(d)
    W = nddo.local_to_tensor(nddo.local_eri(R, ea, eb))[0]
    c = nddo.E2 / Rl
    assert W[0, 0, 0, 0] == pytest.approx(c, rel=1e-6)
    assert W[1, 1, 0, 0] == pytest.approx(c, rel=1e-6)
    assert W[3, 3, 2, 2] == pytest.approx(c, rel=1e-6)
    assert abs(W[0, 3, 0, 0]) < 1e-3 * c
    assert abs(W[1, 3, 1, 3]) < 1e-5 * c


def _block_rotation(sysm, rot):
    T = np.zeros((sysm.n, sysm.n))
    k = 0
    for A in range(sysm.N):
        T[k, k] = 1.0
        if sysm.norb_atom[A] == 4:
            T[k + 1:k + 4, k + 1:k + 4] = rot
        k += sysm.norb_atom[A]
    return T


def test_rotational_invariance_of_fock_and_energy():
    """F(rot R, T P T^T) = T F(R, P) T^T: pins the rotation and the xy-relation."""
    mol = synth.c4h6(1)
    sysm = ham.System(mol.Z, TAB)
    rng = np.random.default_rng(3)
    P = rng.normal(size=(sysm.n, sysm.n)) * 0.1
    P = P + P.T
    a, b, c = 0.3, -1.1, 0.7
    Rx = np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])
    Ry = np.array([[math.cos(b), 0, math.sin(b)], [0, 1, 0], [-math.sin(b), 0, math.cos(b)]])
    Rz = np.array([[math.cos(c), -math.sin(c), 0], [math.sin(c), math.cos(c), 0], [0, 0, 1]])
    rot = Rz @ Ry @ Rx
    T = _block_rotation(sysm, rot)
    F1, h1, G1, V1 = ham.fock(sysm, mol.R, P)
    F2, h2, G2, V2 = ham.fock(sysm, mol.R @ rot.T + np.array([0.3, -2.0, 1.0]), T @ P @ T.T)
    assert np.abs(F2 - T @ F1 @ T.T).max() < 1e-10
    assert V2 == pytest.approx(V1, rel=1e-13)


def test_complex_step_matches_finite_difference():
    d, ea, eb = _pair(6, 7, 1.45, direction=(0.3, -0.5, 0.8))
    W, S, E, dW, dS, dE = nddo.pair_derivatives(d, ea, eb)
    h = 1e-5
    for k in range(3):
        dp, dm = d.copy(), d.copy()
        dp[0, k] += h
        dm[0, k] -= h
        Wp, Sp, Ep = nddo.pair_values(dp, ea, eb)
        Wm, Sm, Em = nddo.pair_values(dm, ea, eb)
        assert np.abs((Wp - Wm) / (2 * h) - dW[:, k]).max() < 1e-6
        assert np.abs((Sp - Sm) / (2 * h) - dS[:, k]).max() < 1e-8
        assert abs((Ep - Em)[0] / (2 * h) - dE[0, k]) < 1e-6
