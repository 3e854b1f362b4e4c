"""Oracle: NDDO integrals over atom pairs (MNDO multipole form, AM1 core-core).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper fixes the Hamiltonian family (AM1/MNDO/PM3 NDDO, Introduction; S = I
under eq. 6) but prints no integral formula.  This module is the MNDO
point-charge multipole model written out from its definition:

* every orbital product on an atom is a set of point charges in the pair's
  local frame (z' from A to B): ss -> monopole; s p_k -> dipole +-1/2 at +-D1
  e_k; p_k p_k -> monopole + linear quadrupole (+1/4 at +-2 D2 e_k, -1/2 at 0);
  p_k p_l -> square quadrupole (+-1/4 at +-D2 e_k +-D2 e_l);
* two charges q_i (atom A, additive term rho_i) and q_j (atom B, rho_j)
  interact as e^2 q_i q_j / sqrt(r_ij^2 + (rho_i + rho_j)^2);
* D1 = <s|z|p_z>, D2^2 = <p|r^2|p>/5 for Slater orbitals; the additive terms
  rho0, rho1, rho2 make the one-centre limits G_ss, H_sp, H_pp exact (rho2
  from the square-quadrupole self interaction, a reading);
* (p_pi p_pi'|p_pi p_pi') = [(p_pi p_pi|p_pi p_pi) - (p_pi p_pi|p_pi' p_pi')]/2
  so that the rotated integrals do not depend on the choice of x' (MNDO's
  rotational-invariance relation);
* molecular-frame integrals are the local ones rotated index by index;
* resonance h_mu,lam = (beta_mu + beta_lam) S_mu,lam / 2 with S the Slater
  overlap, evaluated in prolate spheroidal coordinates;
* core-core: Z'_A Z'_B (ss|ss)(1 + e^{-alpha_A R} + e^{-alpha_B R}) plus AM1
  Gaussians (Z'_A Z'_B / R) sum_k a_k exp(-b_k (R - c_k)^2) for A and B.

Derivatives with respect to the pair vector d = R_B - R_A are taken by the
complex-step method (exact to rounding, independent of any hand derivation).

Pins (tests/test_oracle_nddo.py): 1s-1s overlap closed form, overlaps vs 3-D
quadrature, R -> 0 and R -> infinity limits, rotational invariance, complex
step vs finite differences.  (tests/test_oracle_multipoles_corecore.py): the
charge sets reproduce the monopole, dipole and traceless quadrupole of every
Slater orbital product (radial and angular quadrature); the far field follows
those moments; integrals at bonding distances equal a direct 3-D charge sum;
the core-core term reduces to Z'Z'(ss|ss) (x1, x2, x3 with the exponentials
off / half on / on), decays at each atom's own alpha, carries both atoms'
Gaussians with 1/R, is symmetric in A and B and tends to Z'Z'e^2/R.  Parity
with MOPAC/PySeQM values: unpinned (synthetic parameters, no printed example).
"""
import math
import numpy as np
from scipy.optimize import brentq

E2 = 14.399645          # e^2/(4 pi eps0) in eV*Angstrom
BOHR = 0.52917721090    # Angstrom
H_STEP = 1e-30          # complex-step size (Angstrom)

# orbital slots: 0 = s, 1 = p_x, 2 = p_y, 3 = p_z
PRODUCTS = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (2, 2), (3, 3), (1, 2), (1, 3), (2, 3)]
PROD_INDEX = {}
for _i, (_a, _b) in enumerate(PRODUCTS):
    PROD_INDEX[(_a, _b)] = _i
    PROD_INDEX[(_b, _a)] = _i


# --------------------------------------------------------------------------
# per-element derived parameters
# --------------------------------------------------------------------------
def element_derived(rec):
    """Multipole lengths D1, D2 (Angstrom) and additive terms rho0..2 (Angstrom)."""
    n = int(rec["nprin"])
    norb = int(rec["norb"])
    G_ss, H_sp = rec["G_ss"], rec["H_sp"]
    H_pp = 0.5 * (rec["G_pp"] - rec["G_p2"])
    rho0 = E2 / (2.0 * G_ss) if G_ss > 0 else np.inf
    if norb == 1:
        return dict(D1=0.0, D2=0.0, rho0=rho0, rho1=rho0, rho2=rho0, H_pp=H_pp)
    zs, zp = rec["zeta_s"], rec["zeta_p"]
    D1 = ((2 * n + 1) * (4.0 * zs * zp) ** (n + 0.5)
          / ((zs + zp) ** (2 * n + 2) * math.sqrt(3.0))) * BOHR
    D2 = math.sqrt((4 * n * n + 6 * n + 2) / 20.0) / zp * BOHR

    def dip(r):
        return 0.25 * E2 * (1.0 / r - 1.0 / math.sqrt(D1 * D1 + r * r)) - H_sp

    def quad(r):
        return 0.125 * E2 * (1.0 / r - 2.0 / math.sqrt(D2 * D2 + r * r)
                             + 1.0 / math.sqrt(2.0 * D2 * D2 + r * r)) - H_pp

    rho1 = brentq(dip, 1e-8, 1e3, xtol=1e-15, rtol=1e-15, maxiter=500) if H_sp > 0 else np.inf
    rho2 = brentq(quad, 1e-8, 1e3, xtol=1e-15, rtol=1e-15, maxiter=500) if H_pp > 0 else np.inf
    return dict(D1=D1, D2=D2, rho0=rho0, rho1=rho1, rho2=rho2, H_pp=H_pp)


def one_center_tensor(rec):
    """(mu nu|lam sig) on one atom from G_ss, G_sp, G_pp, G_p2, H_sp, H_pp."""
    I = np.zeros((4, 4, 4, 4))
    H_pp = 0.5 * (rec["G_pp"] - rec["G_p2"])
    I[0, 0, 0, 0] = rec["G_ss"]
    if int(rec["norb"]) == 1:
        return I
    for k in range(1, 4):
        I[0, 0, k, k] = I[k, k, 0, 0] = rec["G_sp"]
        I[k, k, k, k] = rec["G_pp"]
        for a, b in ((0, k), (k, 0)):
            for c, d in ((0, k), (k, 0)):
                I[a, b, c, d] = rec["H_sp"]
        for l in range(1, 4):
            if l != k:
                I[k, k, l, l] = rec["G_p2"]
                for a, b in ((k, l), (l, k)):
                    for c, d in ((k, l), (l, k)):
                        I[a, b, c, d] = H_pp
    return I


# --------------------------------------------------------------------------
# point-charge distributions in the local frame
# --------------------------------------------------------------------------
def _charges(prod, D1, D2, r0, r1, r2):
    """List of (q, (x, y, z), rho) for one orbital product on one atom."""
    a, b = PRODUCTS[prod]
    zero = 0.0 * D1
    if a == 0 and b == 0:
        return [(1.0, (zero, zero, zero), r0)]
    if a == 0:
        e = [zero, zero, zero]
        e_neg = [zero, zero, zero]
        e[b - 1] = D1
        e_neg[b - 1] = -D1
        return [(0.5, tuple(e), r1), (-0.5, tuple(e_neg), r1)]
    if a == b:
        p = [zero, zero, zero]
        m = [zero, zero, zero]
        p[a - 1] = 2.0 * D2
        m[a - 1] = -2.0 * D2
        return [(1.0, (zero, zero, zero), r0), (0.25, tuple(p), r2),
                (0.25, tuple(m), r2), (-0.5, (zero, zero, zero), r2)]
    out = []
    for sa, sb in ((1, 1), (-1, -1), (1, -1), (-1, 1)):
        v = [zero, zero, zero]
        v[a - 1] = sa * D2
        v[b - 1] = sb * D2
        out.append((0.25 * sa * sb, tuple(v), r2))
    return out


def local_eri(R, pa, pb):
    """Local-frame (mu nu|lam sig) for pairs, shape (npair, 10, 10).

    ``R`` may be complex (complex-step derivatives); ``pa``/``pb`` are dicts of
    per-pair arrays D1, D2, rho0, rho1, rho2 for atoms A and B.
    """
    npair = R.shape[0]
    I = np.zeros((npair, 10, 10), dtype=R.dtype)
    ca = [_charges(k, pa["D1"], pa["D2"], pa["rho0"], pa["rho1"], pa["rho2"]) for k in range(10)]
    cb = [_charges(k, pb["D1"], pb["D2"], pb["rho0"], pb["rho1"], pb["rho2"]) for k in range(10)]
    for i in range(10):
        for j in range(10):
            acc = np.zeros(npair, dtype=R.dtype)
            for qa, (xa, ya, za), ra in ca[i]:
                for qb, (xb, yb, zb), rb in cb[j]:
                    dz = za - (zb + R)
                    acc = acc + qa * qb / np.sqrt((xa - xb) ** 2 + (ya - yb) ** 2 + dz * dz
                                                  + (ra + rb) ** 2)
            I[:, i, j] = E2 * acc
    # rotational-invariance relation for (p_x p_y | p_x p_y)
    xx, yy, xy = PROD_INDEX[(1, 1)], PROD_INDEX[(2, 2)], PROD_INDEX[(1, 2)]
    I[:, xy, xy] = 0.5 * (I[:, xx, xx] - I[:, xx, yy])
    return I


def local_to_tensor(I10):
    """(npair, 10, 10) product-indexed integrals -> (npair, 4, 4, 4, 4)."""
    idx = np.array([[PROD_INDEX[(a, b)] for b in range(4)] for a in range(4)])
    return I10[:, idx[:, :, None, None], idx[None, None, :, :]]


# --------------------------------------------------------------------------
# Slater overlaps (prolate spheroidal coordinates)
# --------------------------------------------------------------------------
def _poly_mul(a, b):
    out = np.zeros((a.shape[0] + b.shape[0] - 1, a.shape[1] + b.shape[1] - 1))
    for i in range(a.shape[0]):
        for j in range(a.shape[1]):
            if a[i, j] != 0.0:
                out[i:i + b.shape[0], j:j + b.shape[1]] += a[i, j] * b
    return out


def _poly(terms):
    """Polynomial in (xi, eta) from {(i, j): coeff}."""
    deg_i = max(i for i, _ in terms) + 1
    deg_j = max(j for _, j in terms) + 1
    p = np.zeros((deg_i, deg_j))
    for (i, j), c in terms.items():
        p[i, j] += c
    return p


_XI_P_ETA = _poly({(1, 0): 1.0, (0, 1): 1.0})     # r_A / (R/2)
_XI_M_ETA = _poly({(1, 0): 1.0, (0, 1): -1.0})    # r_B / (R/2)
_ONE = _poly({(0, 0): 1.0})


def _pow(p, k):
    out = _ONE
    for _ in range(k):
        out = _poly_mul(out, p)
    return out


def _overlap_poly(nA, kindA, nB, kindB):
    """Integrand polynomial (without the exponential) and the phi factor.

    kind: 's', 'sig' (p along +z'), 'pi' (p along x').
    """
    vol = _poly({(2, 0): 1.0, (0, 2): -1.0})
    if kindA == "pi":
        radA = _pow(_XI_P_ETA, nA - 2)
        radB = _pow(_XI_M_ETA, nB - 2)
        perp = _poly_mul(_poly({(2, 0): 1.0, (0, 0): -1.0}), _poly({(0, 0): 1.0, (0, 2): -1.0}))
        return _poly_mul(_poly_mul(_poly_mul(vol, radA), radB), perp), math.pi
    if kindA == "s":
        pa = _pow(_XI_P_ETA, nA - 1)
    else:
        pa = _poly_mul(_pow(_XI_P_ETA, nA - 2), _poly({(0, 0): 1.0, (1, 1): 1.0}))
    if kindB == "s":
        pb = _pow(_XI_M_ETA, nB - 1)
    else:
        pb = _poly_mul(_pow(_XI_M_ETA, nB - 2), _poly({(1, 1): 1.0, (0, 0): -1.0}))
    return _poly_mul(_poly_mul(vol, pa), pb), 2.0 * math.pi


def _A_int(p, kmax):
    """A_k(p) = int_1^inf xi^k e^{-p xi} dxi, k = 0..kmax."""
    out = [np.exp(-p) / p]
    for k in range(1, kmax + 1):
        out.append((np.exp(-p) + k * out[-1]) / p)
    return out


def _B_int(q, kmax):
    """B_k(q) = int_{-1}^{1} eta^k e^{-q eta} deta, k = 0..kmax (series for small |q|)."""
    q = np.asarray(q)
    small = np.abs(q.real) < 2.0
    out = []
    # series: sum_m (-q)^m / m! * int eta^{k+m}
    ser = []
    for k in range(kmax + 1):
        acc = np.zeros_like(q)
        term = np.ones_like(q)
        for m in range(40):
            if (k + m) % 2 == 0:
                acc = acc + term * (2.0 / (k + m + 1))
            term = term * (-q) / (m + 1)
        ser.append(acc)
    qs = np.where(small, 1.0, q)
    rec = [(np.exp(qs) - np.exp(-qs)) / qs]
    for k in range(1, kmax + 1):
        rec.append((((-1) ** k) * np.exp(qs) - np.exp(-qs) + k * rec[-1]) / qs)
    for k in range(kmax + 1):
        out.append(np.where(small, ser[k], rec[k]))
    return out


def _norm(n, zeta):
    return (2.0 * zeta) ** (n + 0.5) / math.sqrt(math.factorial(2 * n))


def sto_overlap(R, nA, zA, kindA, nB, zB, kindB):
    """Overlap <chi_A|chi_B> of normalised real Slater orbitals, B at +R z'.

    R in Angstrom (may be complex), zeta in 1/bohr.
    """
    Rb = R / BOHR
    poly, phi = _overlap_poly(nA, kindA, nB, kindB)
    p = 0.5 * Rb * (zA + zB)
    q = 0.5 * Rb * (zA - zB)
    A = _A_int(p, poly.shape[0] - 1)
    B = _B_int(q, poly.shape[1] - 1)
    acc = 0.0
    for i in range(poly.shape[0]):
        for j in range(poly.shape[1]):
            if poly[i, j] != 0.0:
                acc = acc + poly[i, j] * A[i] * B[j]
    ang = {"s": 1.0 / math.sqrt(4 * math.pi), "sig": math.sqrt(3.0 / (4 * math.pi)),
           "pi": math.sqrt(3.0 / (4 * math.pi))}
    pref = _norm(nA, zA) * _norm(nB, zB) * ang[kindA] * ang[kindB] * phi
    return pref * (0.5 * Rb) ** (nA + nB + 1) * acc


# --------------------------------------------------------------------------
# pair blocks in the molecular frame
# --------------------------------------------------------------------------
def local_frame(d):
    """Rotation T (npair, 4, 4): T[k, j] = (e'_j)_k for p slots, T[0, 0] = 1."""
    R = np.sqrt(np.sum(d * d, axis=1))
    u = d / R[:, None]
    ref = np.argmin(np.abs(u.real), axis=1)
    a = np.zeros_like(u)
    a[np.arange(len(u)), ref] = 1.0
    au = np.sum(a * u, axis=1)
    ex = (a - au[:, None] * u) / np.sqrt(1.0 - au * au)[:, None]
    ey = np.cross(u, ex)
    T = np.zeros((len(u), 4, 4), dtype=d.dtype)
    T[:, 0, 0] = 1.0
    T[:, 1:, 1] = ex
    T[:, 1:, 2] = ey
    T[:, 1:, 3] = u
    return R, T


def pair_values(d, ea, eb):
    """Molecular-frame pair quantities for pair vectors d = R_B - R_A.

    ``ea``/``eb`` are dicts of per-pair arrays (element parameters of A and B,
    raw and derived).  Returns W (npair,4,4,4,4) two-centre ERIs with the
    (mu nu) on A and (lam sig) on B, S (npair,4,4) overlaps <A mu|B lam>, and
    Enn (npair,) core-core repulsion.
    """
    R, T = local_frame(d)
    Wloc = local_to_tensor(local_eri(R, ea, eb))
    W = np.einsum("pai,pijkl->pajkl", T, Wloc)
    W = np.einsum("pbj,pajkl->pabkl", T, W)
    W = np.einsum("pck,pabkl->pabcl", T, W)
    W = np.einsum("pdl,pabcl->pabcd", T, W)

    Sloc = np.zeros((len(R), 4, 4), dtype=d.dtype)
    nA, nB = ea["nprin"], eb["nprin"]
    zsA, zpA, zsB, zpB = ea["zeta_s"], ea["zeta_p"], eb["zeta_s"], eb["zeta_p"]
    for key in np.unique(np.stack([nA, nB], axis=1), axis=0):
        sel = (nA == key[0]) & (nB == key[1])
        na_, nb_ = int(key[0]), int(key[1])
        Rs = R[sel]
        Sloc[sel, 0, 0] = sto_overlap(Rs, na_, zsA[sel], "s", nb_, zsB[sel], "s")
        if na_ > 1:
            Sloc[sel, 3, 0] = sto_overlap(Rs, na_, zpA[sel], "sig", nb_, zsB[sel], "s")
        if nb_ > 1:
            Sloc[sel, 0, 3] = sto_overlap(Rs, na_, zsA[sel], "s", nb_, zpB[sel], "sig")
        if na_ > 1 and nb_ > 1:
            Sloc[sel, 3, 3] = sto_overlap(Rs, na_, zpA[sel], "sig", nb_, zpB[sel], "sig")
            spp = sto_overlap(Rs, na_, zpA[sel], "pi", nb_, zpB[sel], "pi")
            Sloc[sel, 1, 1] = spp
            Sloc[sel, 2, 2] = spp
    S = np.einsum("pai,pij,pbj->pab", T, Sloc, T)

    gss = Wloc[:, 0, 0, 0, 0]
    zz = ea["zcore"] * eb["zcore"]
    Enn = zz * gss * (1.0 + np.exp(-ea["alpha"] * R) + np.exp(-eb["alpha"] * R))
    gauss = 0.0
    for e in (ea, eb):
        for k in range(2):
            gauss = gauss + e[f"gauss_a{k}"] * np.exp(-e[f"gauss_b{k}"] * (R - e[f"gauss_c{k}"]) ** 2)
    Enn = Enn + zz / R * gauss
    return W, S, Enn


def pair_derivatives(d, ea, eb):
    """Values and d/d(d_k) of W, S, Enn by the complex-step method.

    Returns (W, S, Enn, dW (npair,3,4,4,4,4), dS (npair,3,4,4), dEnn (npair,3)).
    """
    W, S, Enn = pair_values(d.astype(np.float64), ea, eb)
    dW = np.empty((d.shape[0], 3) + W.shape[1:])
    dS = np.empty((d.shape[0], 3) + S.shape[1:])
    dE = np.empty((d.shape[0], 3))
    for k in range(3):
        dc = d.astype(np.complex128)
        dc[:, k] += 1j * H_STEP
        Wc, Sc, Ec = pair_values(dc, ea, eb)
        dW[:, k] = Wc.imag / H_STEP
        dS[:, k] = Sc.imag / H_STEP
        dE[:, k] = Ec.imag / H_STEP
    return W, S, Enn, dW, dS, dE
