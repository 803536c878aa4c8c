"""Pins of the lambda_1 term of the Israel-Stewart equation (Eq. pimn) and of
the configurable tau_pi, against the second-order viscous Gubser solution
(Sec. 5) and an independent evaluation of the projected pi.pi tensor in full
Milne components."""
import numpy as np
import pytest

import oracle
from conftest import assert_regulator_inactive
from paper_1802_04449_gb300 import inputs as I

HBARC = 0.1973269804


def test_analytic_solution_is_transverse_traceless_and_has_the_ideal_limit():
    x = np.linspace(-3, 3, 13)
    for tau in (1.0, 1.7, 2.5):
        e, ux, uy, pi = I.gubser_viscous(tau, x, x)
        ut = np.sqrt(1 + ux ** 2 + uy ** 2)
        scale = np.abs(pi).max()
        assert np.abs(pi[0] - pi[4] - pi[7] - pi[9]).max() <= 1e-13 * scale
        for row in ((0, 1, 2), (1, 4, 5), (2, 5, 7)):
            t = ut * pi[row[0]] - ux * pi[row[1]] - uy * pi[row[2]]
            assert np.abs(t).max() <= 1e-13 * scale
        # pi~^{eta eta} = 2 eps / lambda1_hat and pi^{xx} = pi^{yy} = -eps / lambda1_hat at r = 0
        c = len(x) // 2
        assert pi[9][c, c] == pytest.approx(2 * e[c, c] / -10.0, rel=1e-13)
        assert pi[4][c, c] == pytest.approx(-e[c, c] / -10.0, rel=1e-13)
    e1, _, _, _ = I.gubser_viscous(1.5, x, x, L=1.0, lambda1_hat=-1e12)
    e2, _, _ = I.gubser_ideal(1.5, x, x, q=1.0)
    np.testing.assert_allclose(e1, e2, rtol=1e-10)


def _milne_X(tau, u, pi):
    """Delta^{mu nu}_{ab} pi^a_l pi^{bl} with the Milne metric, from tilde
    inputs, returned tilde-scaled (tau^{n_mu + n_nu})."""
    n = np.array([0, 0, 0, 1])
    g = np.diag([1.0, -1.0, -1.0, -tau * tau])
    gi = np.linalg.inv(g)
    U = np.array([u[0], u[1], u[2], u[3] / tau])
    idx = [[0, 1, 2, 3], [1, 4, 5, 6], [2, 5, 7, 8], [3, 6, 8, 9]]
    P = np.array([[pi[idx[a][b]] / tau ** (n[a] + n[b]) for b in range(4)] for a in range(4)])
    Y = P @ g @ P
    Ul = g @ U
    D_mix = np.eye(4) - np.outer(U, Ul)          # Delta^mu_a
    D_up = gi - np.outer(U, U)
    D_dn = g - np.outer(Ul, Ul)
    X = D_mix @ Y @ D_mix.T - D_up * np.sum(D_dn * Y) / 3.0
    return np.array([X[a, b] * tau ** (n[a] + n[b]) for a, b in
                     ((0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3))])


@pytest.mark.parametrize("b", [5.0, 44.4])
def test_lambda1_term_equals_the_projected_product(b):
    rng = np.random.default_rng(3)
    lam = -7.5
    o0 = oracle.Oracle(3, 3, 3, 0.2, 0.2, 0.2, 0.6, 0.01, 0.2, None, taupi_coef=b)
    o1 = oracle.Oracle(3, 3, 3, 0.2, 0.2, 0.2, 0.6, 0.01, 0.2, None, taupi_coef=b, lambda1_hat=lam)
    for _ in range(20):
        tau = rng.uniform(0.5, 3.0)
        us = rng.uniform(-0.7, 0.7, 3)
        u = np.concatenate([[np.sqrt(1 + us @ us)], us])
        du = rng.normal(size=16) * 0.3
        pi = rng.normal(size=10)          # neither transverse nor traceless: the full projector matters
        e = rng.uniform(0.5, 20.0)
        T = o1.eos(e)[1]
        inv_taupi = T / (b * 0.2 * HBARC)
        got = o1.source_pi(tau, u, du, pi, e) - o0.source_pi(tau, u, du, pi, e)
        want = -(lam / e) * inv_taupi * _milne_X(tau, u, pi)
        np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12 * np.abs(want).max())


def _gubser_error(dx, lambda1_oracle, b=None, tau1=1.5):
    nx = int(round(8.0 / dx)) + 1
    case = I.gubser_viscous_case(dx=dx, nx=nx, neta=3, deta=0.2, dtau=dx / 20, tau1=tau1)
    o = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                      case.eta_over_s, None, taupi_coef=b or case.taupi_coef, lambda1_hat=lambda1_oracle)
    o.set_initial(case.eps, case.ux, case.uy, case.ueta, case.pi0)
    o.step(case.nsteps)
    if lambda1_oracle == -10.0 and b is None:
        f = o.fields()
        assert_regulator_inactive(f, f["eps"] / 3)
    x = I.cell_coords(nx, dx)
    e, ux, uy, pi = I.gubser_viscous(tau1, x, x, 2.0, -10.0)
    X, Y = np.meshgrid(x, x, indexing="ij")
    core = np.sqrt(X * X + Y * Y) <= 2.0      # out of reach of the edges by tau = 1.5
    err = lambda a, r: np.abs(a[core] - r[core]).mean() / np.abs(r[core]).mean()
    return {k: err(o.get(k)[:, :, 1], r) for k, r in (("eps", e), ("ux", ux), ("pixx", pi[4]), ("piee", pi[9]))}


def test_viscous_gubser_flow_converges():
    """L = 2 fm, eta/s = 0.2, lambda1_hat = -10, tau_pi from the constraint
    (the paper's parameters); tau 1 -> 1.5 fm; L1 errors in r <= 2 fm."""
    e2 = _gubser_error(0.2, -10.0)
    e1 = _gubser_error(0.1, -10.0)
    for k in e1:
        assert e1[k] < 6e-3, (k, e1[k])
        assert e2[k] / e1[k] > 1.9, (k, e2[k], e1[k])


def test_viscous_gubser_pin_needs_the_lambda1_term_and_tau_pi():
    """The same run without the lambda_1 term, with its sign flipped, or with
    the default tau_pi misses the analytic shear stress by an order of
    magnitude more."""
    good = _gubser_error(0.1, -10.0)
    for bad in (_gubser_error(0.1, 0.0), _gubser_error(0.1, 10.0), _gubser_error(0.1, -10.0, b=5.0)):
        assert bad["pixx"] > 8 * good["pixx"] and bad["piee"] > 8 * good["piee"], (bad, good)
