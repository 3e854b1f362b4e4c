"""Oracle: core Hamiltonian, Fock matrix, shadow energy and forces.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* h (eq. 6): one-centre U_mu on the diagonal, electron-core attraction
  -Z'_B (mu nu|s_B s_B) summed over B on diagonal blocks, resonance
  (beta_mu + beta_lam) S_mu,lam / 2 on off-diagonal blocks (NDDO, S = I).
* G(P) = 2J(P) - K(P) (eq. 3), i.e. G_mu,nu = sum_{lam,sig} P_lam,sig
  [2 (mu nu|lam sig) - (mu lam|nu sig)] over the NDDO-allowed integrals;
  F(X) = h + G(X S^-1) with S = I (eq. 17).  P is the per-spin density.
* shadow energy (eq. 13 with the -2 T_e S reading):
  U = 2 Tr[h D] + Tr[(2D - P) G(P)] - 2 T_e S(f) + V_nn.
* forces (eqs. 22, 37-41 with S = I so the Pulay term vanishes):
  dU/dR_I = 2 Tr[h_R D] + Tr[(2D - P) G_R(P)] + dV_nn/dR_I at fixed P,
  F_I = -dU/dR_I (eq. 9 sign; eq. 24 is printed without it).

* dipole moment (Results: the methanol IR spectrum comes from the dipole's
  autocorrelation; the paper does not print its formula).  Reading: the
  NDDO dipole of the point nuclear cores and the valence density with the
  on-site position operator of the zero-differential-overlap basis,
  <mu_A| r |nu_A> = R_A delta_mu,nu plus D1_A for s_A and p_k,A (D1 = <s|z|p_z>),
  so mu = sum_A Z'_A R_A - sum_mu,nu P_mu,nu <mu| r |nu> with P = 2D:
  mu = sum_A (Z'_A - 2 sum_{mu in A} D_mu,mu) R_A - 4 sum_A D1_A (D_s,px, D_s,py, D_s,pz)_A
  in e Angstrom.  Pins: Hellmann-Feynman, mu = -dOmega/dE_field of the SCF
  free energy with the field term added to h, by central differences; a
  neutral molecule's dipole does not depend on the origin, an ion's moves by
  its charge times the shift (tests/test_oracle_dipole.py).

Everything is held in a padded layout with four orbital slots per atom
(hydrogen uses only slot 0); ``orb`` maps the compact n orbitals to slots.
Pins: tests/test_oracle_hamiltonian.py (textbook NDDO Fock form, G = 0,
symmetry, translation/rotation invariance, forces vs finite differences).
"""
import numpy as np

from . import nddo

_FIELDS = ("nprin", "norb", "zcore", "zeta_s", "zeta_p", "alpha",
           "gauss_a0", "gauss_b0", "gauss_c0", "gauss_a1", "gauss_b1", "gauss_c1")


class System:
    """Atoms, parameters, orbital map and pair list of one molecule."""

    def __init__(self, Z, table, charge=0, chunk=4096):
        self.Z = np.asarray(Z, dtype=np.int64)
        self.N = len(self.Z)
        self.table = table
        self.charge = int(charge)
        self.chunk = chunk
        recs = [table[int(z)] for z in self.Z]
        self.rec = recs
        der = {int(z): nddo.element_derived(table[int(z)]) for z in set(self.Z.tolist())}
        self.elem = {}
        for f in _FIELDS:
            self.elem[f] = np.array([r[f] for r in recs], dtype=np.float64)
        for f in ("D1", "D2", "rho0", "rho1", "rho2"):
            self.elem[f] = np.array([der[int(z)][f] for z in self.Z], dtype=np.float64)
        self.norb_atom = self.elem["norb"].astype(np.int64)
        slots = []
        for A in range(self.N):
            slots.extend(4 * A + k for k in range(self.norb_atom[A]))
        self.orb = np.array(slots, dtype=np.int64)          # compact -> padded slot
        self.n = len(self.orb)
        self.nelec = int(round(self.elem["zcore"].sum())) - self.charge
        if self.nelec % 2:
            raise ValueError("open-shell electron count")
        self.nocc = self.nelec // 2
        self.mass = np.array([r["mass"] for r in recs])
        # one-centre data
        self.onec = np.stack([nddo.one_center_tensor(r) for r in recs])      # (N,4,4,4,4)
        U = np.zeros((self.N, 4))
        beta = np.zeros((self.N, 4))
        for A, r in enumerate(recs):
            U[A, 0], beta[A, 0] = r["U_ss"], r["beta_s"]
            if self.norb_atom[A] == 4:
                U[A, 1:], beta[A, 1:] = r["U_pp"], r["beta_p"]
        self.U, self.beta = U, beta
        mask = np.zeros((self.N, 4))
        for A in range(self.N):
            mask[A, : self.norb_atom[A]] = 1.0
        self.mask = mask
        iu = np.triu_indices(self.N, 1)
        self.pA, self.pB = iu[0], iu[1]

    # ---- helpers -------------------------------------------------------
    def pad(self, M):
        P = np.zeros((4 * self.N, 4 * self.N))
        P[np.ix_(self.orb, self.orb)] = M
        return P.reshape(self.N, 4, self.N, 4)

    def unpad(self, Mb):
        return Mb.reshape(4 * self.N, 4 * self.N)[np.ix_(self.orb, self.orb)]

    def _pair_params(self, sel):
        ea = {k: v[self.pA[sel]] for k, v in self.elem.items()}
        eb = {k: v[self.pB[sel]] for k, v in self.elem.items()}
        return ea, eb

    def _pair_mask(self, sel):
        ma, mb = self.mask[self.pA[sel]], self.mask[self.pB[sel]]
        m4 = (ma[:, :, None, None, None] * ma[:, None, :, None, None]
              * mb[:, None, None, :, None] * mb[:, None, None, None, :])
        m2 = ma[:, :, None] * mb[:, None, :]
        return m4, m2

    def chunks(self):
        npair = len(self.pA)
        for s in range(0, npair, self.chunk):
            yield np.arange(s, min(npair, s + self.chunk))


def pair_data(sysm, R, sel, deriv=False):
    """Pair blocks for the pair indices ``sel`` at positions R (N,3)."""
    d = R[sysm.pB[sel]] - R[sysm.pA[sel]]
    ea, eb = sysm._pair_params(sel)
    m4, m2 = sysm._pair_mask(sel)
    if deriv:
        W, S, E, dW, dS, dE = nddo.pair_derivatives(d, ea, eb)
        return W * m4, S * m2, E, dW * m4[:, None], dS * m2[:, None], dE
    W, S, E = nddo.pair_values(d, ea, eb)
    return W * m4, S * m2, E


class PairCache:
    """Pair blocks at one geometry, kept in memory for small systems.

    Large systems (more than ``limit`` pairs) recompute chunk by chunk so the
    oracle's memory stays bounded; the values are the same either way.
    """

    def __init__(self, sysm, R, limit=400000):
        self.sysm, self.R = sysm, np.array(R, dtype=np.float64)
        self.keep = len(sysm.pA) <= limit
        self._val, self._der = {}, {}

    def values(self):
        for i, sel in enumerate(self.sysm.chunks()):
            if i in self._val:
                yield (sel,) + self._val[i]
                continue
            out = pair_data(self.sysm, self.R, sel)
            if self.keep:
                self._val[i] = out
            yield (sel,) + out

    def derivatives(self):
        for i, sel in enumerate(self.sysm.chunks()):
            if i in self._der:
                yield (sel,) + self._der[i]
                continue
            out = pair_data(self.sysm, self.R, sel, deriv=True)
            if self.keep:
                self._der[i] = out
                self._val[i] = out[:3]
            yield (sel,) + out


def _cache(sysm, R, pairs):
    return pairs if pairs is not None else PairCache(sysm, R)


def core_hamiltonian(sysm, R, pairs=None):
    """h (n x n) and V_nn at positions R."""
    N = sysm.N
    hb = np.zeros((N, 4, N, 4))
    for A in range(N):
        hb[A, :, A, :] = np.diag(sysm.U[A] * sysm.mask[A])
    Vnn = 0.0
    zc = sysm.elem["zcore"]
    for sel, W, S, E in _cache(sysm, R, pairs).values():
        A, B = sysm.pA[sel], sysm.pB[sel]
        VA = -zc[B][:, None, None] * W[:, :, :, 0, 0]
        VB = -zc[A][:, None, None] * W[:, 0, 0, :, :]
        hd = np.zeros((N, 4, 4))
        np.add.at(hd, A, VA)
        np.add.at(hd, B, VB)
        for C in range(N):
            hb[C, :, C, :] += hd[C]
        res = 0.5 * (sysm.beta[A][:, :, None] + sysm.beta[B][:, None, :]) * S
        hb[A, :, B, :] = res
        hb[B, :, A, :] = np.transpose(res, (0, 2, 1))
        Vnn += E.sum()
    return sysm.unpad(hb), Vnn


def two_electron(sysm, R, P, pairs=None):
    """G(P) (n x n) for the per-spin density P (eq. 3 with NDDO integrals)."""
    N = sysm.N
    Pb = sysm.pad(P)
    Gb = np.zeros((N, 4, N, 4))
    Pd = np.stack([Pb[A, :, A, :] for A in range(N)])                 # (N,4,4)
    for A in range(N):
        I = sysm.onec[A]
        Gb[A, :, A, :] += (2.0 * np.einsum("mnls,ls->mn", I, Pd[A])
                           - np.einsum("mlns,ls->mn", I, Pd[A]))
    for sel, W, _, _ in _cache(sysm, R, pairs).values():
        A, B = sysm.pA[sel], sysm.pB[sel]
        JA = 2.0 * np.einsum("pmnls,pls->pmn", W, Pd[B])
        JB = 2.0 * np.einsum("pmnls,pmn->pls", W, Pd[A])
        Gd = np.zeros((N, 4, 4))
        np.add.at(Gd, A, JA)
        np.add.at(Gd, B, JB)
        for C in range(N):
            Gb[C, :, C, :] += Gd[C]
        Pab = Pb[A, :, B, :]                                             # (p,4,4)
        K = -np.einsum("pmnls,pns->pml", W, Pab)
        Gb[A, :, B, :] += K
        Gb[B, :, A, :] += np.transpose(K, (0, 2, 1))
    return sysm.unpad(Gb)


def fock(sysm, R, P, pairs=None):
    """F = h + G(P) (eq. 17 with S = I), plus h, G and V_nn."""
    pairs = _cache(sysm, R, pairs)
    h, Vnn = core_hamiltonian(sysm, R, pairs)
    G = two_electron(sysm, R, P, pairs)
    return h + G, h, G, Vnn


def forces(sysm, R, D, P, pairs=None):
    """F_I = -dU/dR_I at fixed P (eq. 37 with S = I), eV/Angstrom, (N,3)."""
    N = sysm.N
    Db, Pb = sysm.pad(D), sysm.pad(P)
    Ab = 2.0 * Db - Pb
    Dd = np.stack([Db[A, :, A, :] for A in range(N)])
    Pd = np.stack([Pb[A, :, A, :] for A in range(N)])
    Ad = np.stack([Ab[A, :, A, :] for A in range(N)])
    zc = sysm.elem["zcore"]
    F = np.zeros((N, 3))
    for sel, W, S, E, dW, dS, dE in _cache(sysm, R, pairs).derivatives():
        A, B = sysm.pA[sel], sysm.pB[sel]
        # 2 Tr[h_R D]: electron-core on diagonal blocks, resonance off-diagonal
        g = 2.0 * (np.einsum("pkmn,pmn->pk", -zc[B][:, None, None, None] * dW[:, :, :, :, 0, 0], Dd[A])
                   + np.einsum("pkls,pls->pk", -zc[A][:, None, None, None] * dW[:, :, 0, 0, :, :], Dd[B]))
        bsum = 0.5 * (sysm.beta[A][:, :, None] + sysm.beta[B][:, None, :])
        g += 2.0 * 2.0 * np.einsum("pkml,pml->pk", bsum[:, None] * dS, Db[A, :, B, :])
        # Tr[(2D - P) G_R(P)]: Coulomb into diagonal blocks, exchange off-diagonal
        g += 2.0 * np.einsum("pkmnls,pmn,pls->pk", dW, Ad[A], Pd[B])
        g += 2.0 * np.einsum("pkmnls,pmn,pls->pk", dW, Pd[A], Ad[B])
        g -= 2.0 * np.einsum("pkmnls,pml,pns->pk", dW, Ab[A, :, B, :], Pb[A, :, B, :])
        g += dE
        np.add.at(F, A, g)
        np.add.at(F, B, -g)
    return F


def electronic_energy_terms(h, G, D, P):
    """2 Tr[h D] + Tr[(2D - P) G(P)] (eq. 13 without entropy and V_nn)."""
    return 2.0 * np.sum(h * D) + np.sum((2.0 * D - P) * G)


def dipole_operator(sysm, R):
    """On-site position operator of the NDDO basis, (3, n, n), Angstrom:
    R_A,k on every orbital of atom A and D1_A between s_A and p_k,A."""
    N = sysm.N
    R = np.asarray(R, dtype=np.float64)
    M = np.zeros((3, N, 4, N, 4))
    for A in range(N):
        for k in range(3):
            M[k, A, :, A, :] = np.diag(R[A, k] * sysm.mask[A])
            if sysm.norb_atom[A] == 4:
                M[k, A, 0, A, 1 + k] = sysm.elem["D1"][A]
                M[k, A, 1 + k, A, 0] = sysm.elem["D1"][A]
    return np.stack([sysm.unpad(M[k]) for k in range(3)])


def dipole(sysm, R, D):
    """Dipole moment (e Angstrom) of the cores and the per-spin density D."""
    M = dipole_operator(sysm, R)
    R = np.asarray(R, dtype=np.float64)
    nuc = (sysm.elem["zcore"][:, None] * R).sum(axis=0)
    return nuc - 2.0 * np.einsum("kij,ij->k", M, D)

