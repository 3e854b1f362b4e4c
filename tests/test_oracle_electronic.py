"""Pins of the oracle's Fermi density, DMPT (eq. 36) and Krylov kernel (eqs. 31-35)."""
import numpy as np
import pytest

import synth
from oracle import hamiltonian as ham, electronic as el, dynamics as dyn

TAB = synth.synthetic_table(1)
MOL = synth.c4h6(1)


@pytest.fixture(scope="module")
def scf_state():
    sysm = ham.System(MOL.Z, TAB)
    cfg = dyn.Config(Te=1000.0)
    D, _ = dyn.scf(sysm, MOL.R, cfg)
    ev = dyn.evaluate(sysm, MOL.R, D, cfg, krylov=False)
    return sysm, cfg, D, ev


def test_density_invariants(scf_state):
    sysm, cfg, D, ev = scf_state
    D0 = ev["D"]
    assert np.trace(D0) == pytest.approx(sysm.nocc, abs=1e-11)        # eq. 8
    assert np.array_equal(D0, D0.T)
    w = np.linalg.eigvalsh(D0)
    assert w.min() > -1e-12 and w.max() < 1 + 1e-12                     # f in [0, 1]
    assert el.fermi(ev["eps"], ev["mu"], cfg.beta).sum() == pytest.approx(sysm.nocc, abs=1e-11)


def test_idempotent_as_temperature_goes_to_zero(scf_state):
    sysm, cfg, D, ev = scf_state
    F = ev["F"]
    gap = ev["eps"][sysm.nocc] - ev["eps"][sysm.nocc - 1]
    Te = 10.0
    D0 = el.density(F, sysm.nocc, Te)[0]
    beta = 1.0 / (el.KB * Te)
    bound = max(sysm.n * np.exp(-beta * gap / 2), 1e-13)
    assert np.abs(D0 @ D0 - D0).max() <= bound
    # and at 1000 K with a ~10 eV gap the deviation is already tiny
    assert np.abs(ev["D"] @ ev["D"] - ev["D"]).max() < 1e-12


def test_entropy_special_values():
    assert el.entropy([0.5]) == pytest.approx(el.KB * np.log(2.0), rel=1e-15)
    assert el.entropy([0.0, 1.0]) == 0.0
    f = np.array([0.2, 0.7])
    ref = -el.KB * sum(x * np.log(x) + (1 - x) * np.log(1 - x) for x in f)
    assert el.entropy(f) == pytest.approx(ref, rel=1e-15)


@pytest.mark.parametrize("Te", [1000.0, 30000.0])
def test_dmpt_matches_finite_differences(scf_state, Te):
    """D1 = d/dlambda D[F0 + lambda F1] with mu re-solved (eq. 36)."""
    sysm, _, _, ev = scf_state
    F0 = ev["F"]
    rng = np.random.default_rng(7)
    V = rng.normal(size=F0.shape)
    V = V + V.T
    F1 = ham.two_electron(sysm, MOL.R, V)
    D, eps, Q, f, mu = el.density(F0, sysm.nocc, Te)
    beta = 1.0 / (el.KB * Te)
    Lam = el.divided_differences(eps, f, mu, beta)
    D1, _ = el.dmpt(F1, Q, Lam)
    h = 1e-5
    Dp = el.density(F0 + h * F1, sysm.nocc, Te)[0]
    Dm = el.density(F0 - h * F1, sysm.nocc, Te)[0]
    fd = (Dp - Dm) / (2 * h)
    assert np.abs(D1 - fd).max() < 1e-7 * max(1.0, np.abs(D1).max())
    assert abs(np.trace(D1)) < 1e-12
    assert np.array_equal(D1, D1.T)


def test_dmpt_zero_temperature_block_structure(scf_state):
    """T -> 0 with a gap: Lambda vanishes inside the occ/occ and virt/virt blocks."""
    sysm, _, _, ev = scf_state
    Te = 50.0
    D, eps, Q, f, mu = el.density(ev["F"], sysm.nocc, Te)
    Lam = el.divided_differences(eps, f, mu, 1.0 / (el.KB * Te))
    no = sysm.nocc
    assert np.abs(Lam[:no, :no]).max() < 1e-10
    assert np.abs(Lam[no:, no:]).max() < 1e-10
    # occ/virt entries tend to -1/(eps_a - eps_i), the textbook first-order response
    ref = -1.0 / (eps[no:][None, :] - eps[:no][:, None])
    assert np.abs(Lam[:no, no:] - ref).max() < 1e-10


def _response(sysm, ev, beta):
    Lam = el.divided_differences(ev["eps"], ev["f"], ev["mu"], beta)

    def resp(V):
        return el.dmpt(ham.two_electron(sysm, MOL.R, V), ev["Q"], Lam)[0]
    return resp


def test_krylov_full_rank_equals_exact_inverse_jacobian(scf_state):
    """Krylov result at full rank = J^-1 W0 with J built on every symmetric direction."""
    sysm, cfg, D, ev = scf_state
    n = sysm.n
    resp = _response(sysm, ev, cfg.beta)
    iu = np.triu_indices(n)
    basis = []
    for i, j in zip(*iu):
        E = np.zeros((n, n))
        E[i, j] = E[j, i] = 1.0 if i != j else 1.0
        basis.append(E / np.linalg.norm(E))
    Bm = np.stack([b.ravel() for b in basis], axis=1)              # (n^2, dim)
    J = np.stack([((resp(b) - b).ravel()) for b in basis], axis=1)  # J b_k in R^{n^2}
    Jr = Bm.T @ J                                                   # restricted to sym space
    rng = np.random.default_rng(11)
    Y = rng.normal(size=(n, n))
    W0 = 1e-3 * (Y + Y.T)
    exact = (Bm @ np.linalg.solve(Jr, Bm.T @ W0.ravel())).reshape(n, n)
    K, info = el.krylov_kernel(W0, resp, m_max=len(basis))
    assert info["fit"][-1] < 1e-9
    assert np.abs(K - exact).max() < 1e-8 * np.abs(exact).max()


def test_krylov_without_two_electron_terms_is_minus_identity():
    tab0 = synth.synthetic_table(1, two_electron=False)
    sysm = ham.System(MOL.Z, tab0)
    cfg = dyn.Config(Te=1000.0, m=3)
    X = dyn.initial_guess(sysm)
    ev = dyn.evaluate(sysm, MOL.R, X, cfg)
    W0 = ev["D"] - X
    for m in (1, 2, 3):
        K, info = el.krylov_kernel(W0, _response(sysm, ev, cfg.beta), m_max=m)
        assert np.abs(K + W0).max() < 1e-12 * np.abs(W0).max()


def test_krylov_fit_error_monotone_and_normal_equations(scf_state):
    sysm, cfg, D, ev = scf_state
    rng = np.random.default_rng(5)
    Y = rng.normal(size=D.shape)
    X = D + 1e-3 * (Y + Y.T)
    ev2 = dyn.evaluate(sysm, MOL.R, X, cfg, krylov=False)
    W0 = ev2["D"] - X
    K, info = el.krylov_kernel(W0, _response(sysm, ev2, cfg.beta), m_max=8)
    fit = np.array(info["fit"])
    assert np.all(np.diff(fit) <= 1e-14)
    r = sum(c * W for c, W in zip(info["c"], info["W"])) - W0
    for W in info["W"]:
        assert abs(el.inner(W, r)) < 1e-12 * np.linalg.norm(W0) * np.linalg.norm(W)
    V = np.stack([v.ravel() for v in info["V"]])
    assert np.abs(V @ V.T - np.eye(len(V))).max() < 1e-13
