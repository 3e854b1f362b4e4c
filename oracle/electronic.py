"""Oracle: Fermi-Dirac density matrix, entropy, DMPT response, Krylov kernel.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* eq. 19 with S = I (Z = I, eqs. 18, 20, 21): D0 = Q diag(f) Q^T from the
  eigendecomposition F = Q diag(eps) Q^T (LAPACK ``eigh``);
  f_i = 1/(exp(beta (eps_i - mu)) + 1) (eq. 7) with mu fixed by
  sum f_i = N_occ (eq. 8), written as (1 - tanh(beta (eps - mu)/2))/2.
  mu: bisection on [eps_min - 40/beta, eps_max + 40/beta] then Newton
  polish (the paper does not state the solver; a reading).
* eq. 4: S(f) = -k_B sum [f ln f + (1 - f) ln(1 - f)], 0 ln 0 = 0.
* eq. 36: canonical finite-temperature DMPT
  D1 = Q [Lambda o (Q^T F1 Q - dmu I)] Q^T with Lambda_ij =
  (f_i - f_j)/(eps_i - eps_j), Lambda_ii = -beta f_i (1 - f_i) and
  dmu = sum_i Lambda_ii F1'_ii / sum_i Lambda_ii so that Tr D1 = 0 (the
  pseudocode is in the paper's ref. 16; this is the reading).  Pairs with
  beta |eps_i - eps_j| < 1e-5 use the derivative at the midpoint.
* eqs. 31-35: Krylov subspace approximation of K (D0 - X) with K0 = I:
  W0 = D0 - X; V_k = W_{k-1} orthogonalised (classical Gram-Schmidt twice)
  against V_1..V_{k-1} (stop if that removes all but 1e-10 of its norm) and normalised in <A, B> = Tr[A^T B]; W_k = D1[V_k] - V_k
  (directional derivative of the residual, eq. 31 with F1 = G(V_k));
  O_ij = <W_i, W_j>, c = O^-1 b, b_j = <W_j, W0>; result sum_i V_i c_i
  (eq. 34 with M = O^-1).  Adaptive rank: stop when k >= m_min and the
  relative fit error ||sum c_i W_i - W0|| / ||W0|| < tol.

Symmetry: eqs. 19 and 36 define symmetric matrices, but the rounded products
Q diag(f) Q^T and Q Y Q^T are not bitwise symmetric.  An antisymmetric part
of X has no restoring force in eq. 29 and was seen to grow ~1.5x per step
from 1e-17, so D0 and D1 are symmetrised, (A + A^T)/2, after the products;
every Krylov vector and X(t) is then a linear combination of exactly
symmetric matrices.

Pins: tests/test_oracle_electronic.py (trace, symmetry, spectrum in [0,1],
idempotency as T_e -> 0, DMPT vs finite differences, Krylov vs the exact
Jacobian, G = 0 => K = -I, monotone fit error, normal equations).
"""
import numpy as np
import scipy.linalg

KB = 8.617333262e-5   # eV/K


def fermi(eps, mu, beta):
    return 0.5 * (1.0 - np.tanh(0.5 * beta * (eps - mu)))


def chemical_potential(eps, nocc, beta, iters=200):
    """mu with sum_i f_i(mu) = nocc (eq. 8): bisection + Newton polish."""
    lo = eps.min() - 40.0 / beta
    hi = eps.max() + 40.0 / beta
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if fermi(eps, mid, beta).sum() > nocc:
            hi = mid
        else:
            lo = mid
        if hi - lo < 1e-15 * max(1.0, abs(mid)):
            break
    mu = 0.5 * (lo + hi)
    for _ in range(3):
        f = fermi(eps, mu, beta)
        dn = beta * np.sum(f * (1.0 - f))
        if dn < 1e-300:
            break
        step = (nocc - f.sum()) / dn
        if not np.isfinite(step) or abs(step) > 1.0 / beta:
            break
        mu += step
    return mu


def entropy(f):
    """S(f) / k_B-scaled per eq. 4 (returns S in eV/K)."""
    f = np.asarray(f)
    t = np.zeros_like(f)
    m = (f > 0) & (f < 1)
    t[m] = f[m] * np.log(f[m]) + (1.0 - f[m]) * np.log(1.0 - f[m])
    return -KB * t.sum()


def density(F, nocc, Te):
    """D0 = Fermi(F) (eq. 19) with eigenpairs, occupations and mu."""
    beta = 1.0 / (KB * Te)
    eps, Q = scipy.linalg.eigh(F)
    mu = chemical_potential(eps, nocc, beta)
    f = fermi(eps, mu, beta)
    D = (Q * f) @ Q.T
    D = 0.5 * (D + D.T)          # exact symmetry (see module header)
    return D, eps, Q, f, mu


def divided_differences(eps, f, mu, beta, tie=1e-5):
    """Lambda_ij = (f_i - f_j)/(eps_i - eps_j); midpoint derivative for ties."""
    de = eps[:, None] - eps[None, :]
    df = f[:, None] - f[None, :]
    mid = 0.5 * (eps[:, None] + eps[None, :])
    fm = fermi(mid, mu, beta)
    deriv = -beta * fm * (1.0 - fm)
    tie_mask = beta * np.abs(de) < tie
    safe = np.where(tie_mask, 1.0, de)
    return np.where(tie_mask, deriv, df / safe)


def dmpt(F1, Q, Lam):
    """D1 = Q [Lambda o (Q^T F1 Q - dmu I)] Q^T with Tr D1 = 0 (eq. 36)."""
    F1p = Q.T @ F1 @ Q
    ld = np.diag(Lam)
    den = ld.sum()
    dmu = (ld * np.diag(F1p)).sum() / den if abs(den) > 1e-300 else 0.0
    Y = Lam * (F1p - dmu * np.eye(len(ld)))
    D1 = Q @ Y @ Q.T
    return 0.5 * (D1 + D1.T), dmu


def inner(A, B):
    return float(np.sum(A * B))


def krylov_kernel(W0, response, m_max, m_min=None, tol=0.0):
    """Rank-m Krylov approximation of K W0 (eqs. 31-35, K0 = I).

    ``response(V)`` returns D1[V] (eq. 36 with F1 = G(V)).  Returns the
    kernel result sum_i V_i c_i and a dict with the rank, coefficients,
    fit errors and the V/W stacks.
    """
    if m_min is None:
        m_min = m_max
    n0 = np.sqrt(inner(W0, W0))
    info = dict(rank=0, c=np.zeros(0), fit=[], V=[], W=[])
    if n0 < 1e-14:
        return np.zeros_like(W0), info
    V, W = [], []
    c = np.zeros(0)
    v = W0
    for k in range(1, m_max + 1):
        nv0 = np.sqrt(inner(v, v))
        for _ in range(2):
            for Vi in V:
                v = v - inner(Vi, v) * Vi
        nv = np.sqrt(inner(v, v))
        if nv < 1e-10 * nv0:          # Krylov breakdown: subspace is invariant
            break
        v = v / nv
        Wk = response(v) - v
        V.append(v)
        W.append(Wk)
        m = len(V)
        O = np.array([[inner(W[i], W[j]) for j in range(m)] for i in range(m)])
        b = np.array([inner(W[j], W0) for j in range(m)])
        try:
            cf = scipy.linalg.cho_factor(O)
            c = scipy.linalg.cho_solve(cf, b)
        except np.linalg.LinAlgError:
            c = np.linalg.lstsq(O, b, rcond=None)[0]
        fit = np.sqrt(inner(sum(ci * Wi for ci, Wi in zip(c, W)) - W0,
                            sum(ci * Wi for ci, Wi in zip(c, W)) - W0)) / n0
        info["fit"].append(fit)
        if k >= m_min and fit < tol:
            break
        v = Wk
    info.update(rank=len(V), c=c, V=V, W=W)
    K = sum(ci * Vi for ci, Vi in zip(c, V))
    return K, info
