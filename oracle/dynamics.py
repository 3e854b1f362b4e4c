"""Oracle: SCF start, shadow-potential evaluation and damped XL-BOMD steps.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Initial state (Methods section 5): X(t0 - k dt) = D_min for k = 0..k_max,
  D_min from SCF by linear mixing P <- 0.1 P + 0.9 D[P] started from a
  diagonal guess (Results, "SCF Optimization"); convergence here is
  max|D[P] - P| < scf_tol (tighter than the paper's 1e-7 eV energy change).
* evaluate(R, X): F = h + G(X) (eq. 17), D0 (eq. 19), shadow energy (eq. 13
  with -2 T_e S), forces (eq. 37), Krylov kernel of D0 - X (eq. 34).
* step (eqs. 27-30, 35): Rdot(t+dt/2) = Rdot + dt/2 Rddot;
  R(t+dt) = R + dt Rdot(t+dt/2);
  X(t+dt) = 2X(t) - X(t-dt) - kappa sum V_i c_i + alpha sum_k c_k X(t-k dt);
  evaluate at (R(t+dt), X(t+dt)); Rdot(t+dt) = Rdot(t+dt/2) + dt/2 Rddot(t+dt).
* constant of motion (eq. 26): E_tot = sum M Rdot^2 / 2 + U(R, X).
* comparison mode (Results, Langevin run of C240 2+): the original XL-BOMD
  kernel, a scaled delta function K = -c I, so K (D0 - X) = -c (D0 - X) and
  no response calculation is made (Config.xl_c = c; None selects eq. 34).
  Pin: with every two-electron integral zero the Jacobian of D0 - X is -I, so
  the Krylov kernel at any rank equals the c = 1 kernel exactly.
* Langevin thermostat (Results: Langevin runs at 300 K; the scheme and the
  friction are not printed): reading, the Ornstein-Uhlenbeck half steps of the
  OBABO splitting around the Verlet step, V <- c V + sqrt((1 - c^2) k_B T / M) xi
  with c = exp(-gamma dt / 2), xi from the counter-based generator of rng.py.
* comparison mode (Results, BOMD reusing the previous density): Config.bomd
  re-converges the SCF (linear mixing from the previous density) at every
  new geometry and takes forces at X = D_scf; there is no X dynamics.

The damping constants (kappa, alpha, c_k for k_max = 6) are given in the
paper's ref. 24 and not printed in the paper; the values below are that
reading.  Pins: sum c_k = 0 and sum k c_k = 0 (the damping term vanishes on
a linear trajectory) and every root of the damped recursion with K = -I lies
inside the unit circle (tests/test_oracle_dynamics.py); energy conservation
of the oracle trajectory.
"""
import numpy as np

from . import hamiltonian as ham
from . import electronic as el
from . import rng

KB = el.KB
ACC = 9.648533212e-3          # Angstrom/fs^2 per (eV/Angstrom)/amu
KMAX = 6
KAPPA = 1.84
ALPHA = 0.0055
CK = np.array([-14.0, 36.0, -27.0, -2.0, 12.0, -6.0, 1.0])


class Config:
    def __init__(self, Te=1000.0, dt=0.5, m=4, m_min=None, tol=0.0,
                 scf_tol=1e-10, scf_max=2000, mix=0.1, xl_c=None, bomd=False,
                 langevin_T=300.0, gamma=0.0, seed=0):
        self.Te, self.dt, self.m = Te, dt, m
        self.xl_c = xl_c
        self.bomd = bomd
        self.langevin_T, self.gamma, self.seed = langevin_T, gamma, seed
        self.m_min = m if m_min is None else m_min
        self.tol, self.scf_tol, self.scf_max, self.mix = tol, scf_tol, scf_max, mix

    @property
    def beta(self):
        return 1.0 / (KB * self.Te)


def initial_guess(sysm):
    """Diagonal per-spin guess: valence electrons spread over the atom's orbitals."""
    d = np.zeros(sysm.n)
    k = 0
    for A in range(sysm.N):
        no = sysm.norb_atom[A]
        d[k:k + no] = 0.5 * sysm.elem["zcore"][A] / no
        k += no
    d *= sysm.nocc / d.sum()
    return np.diag(d)


def scf(sysm, R, cfg, P0=None):
    """Linear-mixing SCF: P <- mix P + (1 - mix) D[P] until max|D - P| < tol."""
    P = initial_guess(sysm) if P0 is None else P0.copy()
    pairs = ham.PairCache(sysm, R)
    h, _ = ham.core_hamiltonian(sysm, R, pairs)
    for it in range(cfg.scf_max):
        F = h + ham.two_electron(sysm, R, P, pairs)
        D = el.density(F, sysm.nocc, cfg.Te)[0]
        err = np.abs(D - P).max()
        if err < cfg.scf_tol:
            return D, it
        P = cfg.mix * P + (1.0 - cfg.mix) * D
    raise RuntimeError(f"SCF did not converge (max|D-P| = {err:.3e})")


def scf_krylov(sysm, R, cfg, m, P0=None, tol=None, max_iter=None):
    """Low-rank Krylov SCF (Results, "SCF Optimization": fixed rank, no
    preconditioner).  The SCF residual D[P] - P has the same Jacobian as the
    XL-BOMD residual (eq. 31), so the rank-m kernel of eqs. 31-34 gives the
    Newton-like update P <- P - K (D[P] - P).  Reading: whenever the residual
    has grown tenfold over the best one seen, a linear-mixing step is taken
    instead.  Returns (P, iterations, residual history)."""
    tol = cfg.scf_tol if tol is None else tol
    max_iter = cfg.scf_max if max_iter is None else max_iter
    P = initial_guess(sysm) if P0 is None else P0.copy()
    pairs = ham.PairCache(sysm, R)
    h, _ = ham.core_hamiltonian(sysm, R, pairs)
    best, hist = np.inf, []
    for it in range(max_iter):
        F = h + ham.two_electron(sysm, R, P, pairs)
        D, eps, Q, f, mu = el.density(F, sysm.nocc, cfg.Te)
        err = np.abs(D - P).max()
        hist.append(err)
        if err < tol:
            return D, it, hist
        best = min(best, err)
        if err < 10.0 * best:
            Lam = el.divided_differences(eps, f, mu, cfg.beta)

            def response(V):
                return el.dmpt(ham.two_electron(sysm, R, V, pairs), Q, Lam)[0]

            K, _ = el.krylov_kernel(D - P, response, m, m, 0.0)
            P = P - K
        else:
            P = cfg.mix * P + (1.0 - cfg.mix) * D
    raise RuntimeError(f"Krylov SCF did not converge (max|D-P| = {err:.3e})")


def evaluate(sysm, R, X, cfg, krylov=True):
    """Shadow energy, forces, D0 and Krylov kernel at (R, X)."""
    pairs = ham.PairCache(sysm, R)
    F, h, G, Vnn = ham.fock(sysm, R, X, pairs)
    D, eps, Q, f, mu = el.density(F, sysm.nocc, cfg.Te)
    S = el.entropy(f)
    U = ham.electronic_energy_terms(h, G, D, X) - 2.0 * cfg.Te * S + Vnn
    forces = ham.forces(sysm, R, D, X, pairs)
    out = dict(F=F, h=h, G=G, D=D, eps=eps, Q=Q, f=f, mu=mu, S=S, U=U, Vnn=Vnn,
               forces=forces, Te=cfg.Te)
    if krylov and cfg.xl_c is not None:
        W0 = D - X
        out.update(K=-cfg.xl_c * W0,
                   krylov=dict(rank=0, c=np.zeros(0), fit=[], V=[], W=[]))
    elif krylov:
        Lam = el.divided_differences(eps, f, mu, cfg.beta)

        def response(V):
            return el.dmpt(ham.two_electron(sysm, R, V, pairs), Q, Lam)[0]

        K, info = el.krylov_kernel(D - X, response, cfg.m, cfg.m_min, cfg.tol)
        out.update(K=K, krylov=info, Lam=Lam)
    return out


class State:
    """R, Rdot, X history (X[0] = X(t), X[k] = X(t - k dt)) and last evaluation."""

    def __init__(self, sysm, R, V, cfg, X0=None):
        self.sysm, self.cfg = sysm, cfg
        self.R = np.array(R, dtype=np.float64)
        self.V = np.array(V, dtype=np.float64)
        if X0 is None:
            X0, self.scf_iters = scf(sysm, self.R, cfg)
        self.X = [X0.copy() for _ in range(KMAX + 1)]
        self.ev = evaluate(sysm, self.R, self.X[0], cfg, krylov=not cfg.bomd)
        self.t = 0
        self.scf_iters_last = 0

    @property
    def acc(self):
        return ACC * self.ev["forces"] / self.sysm.mass[:, None]

    def kinetic(self):
        return 0.5 * np.sum(self.sysm.mass[:, None] * self.V ** 2) / ACC

    def total_energy(self):
        return self.kinetic() + self.ev["U"]

    def thermostat(self, phase):
        """Ornstein-Uhlenbeck half step (Langevin, OBABO splitting)."""
        cfg = self.cfg
        c = np.exp(-0.5 * cfg.gamma * cfg.dt)
        sigma = np.sqrt((1.0 - c * c) * KB * cfg.langevin_T * ACC / self.sysm.mass)
        xi = rng.normals(3 * self.sysm.N, phase, self.t, cfg.seed).reshape(-1, 3)
        self.V = c * self.V + sigma[:, None] * xi

    def step(self):
        if self.cfg.gamma > 0.0:
            self.thermostat(0)
            ev = self._verlet_step()
            self.thermostat(1)
            self.t += 1
            return ev
        ev = self._verlet_step()
        self.t += 1
        return ev

    def _verlet_step(self):
        dt = self.cfg.dt
        self.V = self.V + 0.5 * dt * self.acc
        self.R = self.R + dt * self.V
        if self.cfg.bomd:
            P, self.scf_iters_last = scf(self.sysm, self.R, self.cfg, P0=self.X[0])
            self.X = [P] + self.X[:KMAX]
            self.ev = evaluate(self.sysm, self.R, P, self.cfg, krylov=False)
            self.V = self.V + 0.5 * dt * self.acc
            return self.ev
        Xn = 2.0 * self.X[0] - self.X[1] - KAPPA * self.ev["K"]
        Xn = Xn + ALPHA * sum(CK[k] * self.X[k] for k in range(KMAX + 1))
        self.X = [Xn] + self.X[:KMAX]
        self.ev = evaluate(self.sysm, self.R, self.X[0], self.cfg)
        self.V = self.V + 0.5 * dt * self.acc
        return self.ev


def energy_drift(times_fs, etot, natoms):
    """Linear-fit slope of E_tot(t) in eV/ps/atom (Results, Gramicidin S)."""
    slope = np.polyfit(np.asarray(times_fs) * 1e-3, np.asarray(etot), 1)[0]
    return slope / natoms
