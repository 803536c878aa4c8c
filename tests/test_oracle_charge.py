"""Pins of the net-charge transport of the oracle (reading R19: Eq. (Ntilde)
with S_N = 0 and no diffusion current; the paper runs with n = 0):
  - the Gubser closed form for n satisfies d_mu(tau n u^mu) = 0 (checked
    symbolically), and the oracle's evolution converges to it;
  - in a periodic Cartesian box the total charge is conserved to rounding;
  - uniform Bjorken flow keeps n tau constant exactly.
"""
import numpy as np
import pytest

import oracle
from paper_1802_04449_gb300 import inputs as I


def test_gubser_charge_closed_form_is_conserved():
    sp = pytest.importorskip("sympy")
    t, r, q = sp.symbols("tau r q", positive=True)
    v = 2 * q * q * t * r / (1 + q * q * (t * t + r * r))
    g = 1 / sp.sqrt(1 - v ** 2)
    n = 4 * q * q / (t * (1 + 2 * q * q * (t * t + r * r) + q ** 4 * (t * t - r * r) ** 2))
    assert sp.simplify(sp.diff(t * n * g, t) + sp.diff(r * t * n * g * v, r) / r) == 0
    # and the generator evaluates that expression
    x = np.array([0.0, 0.7, 1.9])
    got = I.gubser_charge(1.3, x, np.zeros(1), q=1.0, n_norm=1.0)[:, 0]
    f = sp.lambdify((t, r, q), n)
    np.testing.assert_allclose(got, [f(1.3, xx, 1.0) / f(1.0, 0.0, 1.0) for xx in x], rtol=1e-14)


def gubser_charge_err(dx, tau1=1.6, plant=0):
    half = 4.8
    nx = int(round(2 * half / dx)) + 1
    c = I.gubser_case(dx=dx, nx=nx, neta=1, deta=0.3, dtau=dx / 10, tau1=tau1)
    x = I.cell_coords(c.nx, c.dx)
    o = oracle.Oracle(c.nx, c.ny, 1, c.dx, c.dy, c.deta, c.tau0, c.dtau, plant=plant)
    o.set_initial(c.eps, c.ux, c.uy, c.ueta)
    o.set_initial_n(I.gubser_charge(c.tau0, x, x)[:, :, None])
    o.step(c.nsteps)
    na = I.gubser_charge(o.stats()["tau"], x, x)
    X, Y = np.meshgrid(x, x, indexing="ij")
    m = X ** 2 + Y ** 2 <= 2.5 ** 2
    no = o.get("n")[:, :, 0]
    return np.abs(no - na)[m].sum() / np.abs(na[m]).sum()


def check_gubser_charge(plant=0):
    e1, e2, e3 = (gubser_charge_err(dx, plant=plant) for dx in (0.3, 0.15, 0.075))
    # minmod clips the maximum of n at the centre: the observed order is
    # between 1 and 2 (0.035, 0.019, 0.009)
    assert e3 < 0.012 and e1 > e2 > e3 and e2 / e3 > 1.9 and e1 / e2 > 1.6, (e1, e2, e3)


def test_gubser_charge_converges():
    """Ideal conformal Gubser flow with its conserved charge: L1 error of n
    for r <= 2.5 fm falls under refinement (dx 0.3, 0.15, 0.075)."""
    check_gubser_charge()


def test_total_charge_is_conserved_in_a_periodic_box():
    rng = np.random.default_rng(4)
    nx, ny, ne = 12, 10, 8
    eps, ux, uy, ue = I.random_smooth_box(rng, nx, ny, ne)
    n0 = 0.3 + 0.1 * np.cos(2 * np.pi * np.arange(nx) / nx)[:, None, None] * np.ones((nx, ny, ne))
    o = oracle.Oracle(nx, ny, ne, 0.3, 0.3, 0.3, 0.0, 0.02, cartesian=True, periodic=True)
    o.set_initial(eps, ux, uy, ue)
    o.set_initial_n(n0)
    q0 = o.get("Nt").sum()
    o.step(100)
    q1 = o.get("Nt").sum()
    assert abs(q1 - q0) <= 1e-13 * abs(q0), (q0, q1)
    assert o.get("n").min() > 0


def check_bjorken_charge(plant=0):
    tau0 = 0.6
    o = oracle.Oracle(4, 4, 4, 0.3, 0.3, 0.3, tau0, 0.02, periodic=True, plant=plant)
    o.set_initial(np.full((4, 4, 4), 30.0), np.zeros((4, 4, 4)), np.zeros((4, 4, 4)), np.zeros((4, 4, 4)))
    o.set_initial_n(np.full((4, 4, 4), 0.5))
    np.testing.assert_allclose(o.get("n"), 0.5, rtol=1e-14)
    o.step(50)
    tau = o.stats()["tau"]
    np.testing.assert_allclose(o.get("n"), 0.5 * tau0 / tau, rtol=1e-12)


def test_bjorken_flow_keeps_n_tau_constant():
    check_bjorken_charge()
