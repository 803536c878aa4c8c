"""Pins of the Cooper-Frye oracle (oracle/clv_cooperfrye.c, Sec. 4, Eqs.
(cooper_frye) and (feq), readings C1-C4).  Each is fixed by something other
than the oracle's own formula:
  - a boost-invariant tau = const surface at rest integrates over eta_s to
    the Bessel-function closed form 2 mT sum_n (-s)^(n-1) K_1(n mT / T);
  - the momentum integral of the spectrum of any one element is the number
    of particles n u.dSigma, with n the thermal density of Eq.
    (thermal_density_i) (a one-dimensional quadrature);
  - the pi~ moments of the spectrum of an element at rest are fixed
    one-dimensional integrals of f (1 - s f) (isotropy of the rest frame).
"""
import numpy as np
import pytest
from scipy import integrate, special

import oracle

HBARC = 0.1973269804
M_PI = 0.13957
TF = 0.137
NORM = 1.0 / (2 * np.pi * HBARC) ** 3


def _f(E, stat, T=TF):
    return 1.0 / (np.exp(E / T) + stat)


def _element(tau, eta, dS, u, pi=None):
    r = np.zeros(22)
    r[:4] = dS
    r[4], r[7] = tau, eta
    ut = np.sqrt(1 + np.dot(u, u))
    r[8:12] = [ut, *u]
    if pi is not None:
        r[12:] = pi
    return r


def check_bjorken_bessel(plant=0):
    tau, A, H, deta = 1.7, 1.3, 10.0, 0.01
    etas = -H + (np.arange(int(round(2 * H / deta))) + 0.5) * deta
    rec = np.array([_element(tau, e, [tau * A * deta, 0, 0, 0], [0, 0, 0]) for e in etas])
    Y, pT, phi = np.array([0.0, 0.7]), np.array([0.05, 0.6, 1.8]), np.array([0.4])
    for stat in (-1, 0, 1):
        got = oracle.cooper_frye(rec, Y, pT, phi, M_PI, 1.0, stat, TF, viscous=False, plant=plant)
        mT = np.sqrt(pT ** 2 + M_PI ** 2)
        n = np.arange(1, 80)[:, None]
        coef = (-stat) ** (n - 1) if stat != 0 else (n == 1)
        want = NORM * tau * A * 2 * mT * (coef * special.k1(n * mT / TF)).sum(axis=0)
        for a in range(len(Y)):
            np.testing.assert_allclose(got[a, :, 0], want, rtol=1e-10)


def test_boost_invariant_surface_gives_the_bessel_closed_form():
    check_bjorken_bessel()


def _grid(eta0):
    y, wy = np.polynomial.legendre.leggauss(160)
    Y, wY = eta0 + 9.0 * y, 9.0 * wy
    p, wp = np.polynomial.legendre.leggauss(240)
    pT, wpT = 6.0 * (p + 1), 6.0 * wp       # boosted elements reach e^-15 only near 5 GeV
    nphi = 64
    phi = 2 * np.pi * (np.arange(nphi) + 0.5) / nphi
    wphi = np.full(nphi, 2 * np.pi / nphi)
    return Y, wY, pT, wpT, phi, wphi


def _integrate(spec, wY, pT, wpT, wphi, weight=None):
    w = wY[:, None, None] * (wpT * pT)[None, :, None] * wphi[None, None, :]
    return float((w * spec * (1 if weight is None else weight)).sum())


def _density(stat, mass=M_PI, g=1.0):
    """Eq. (thermal_density_i), GeV^3."""
    v, _ = integrate.quad(lambda p: p * p * _f(np.sqrt(p * p + mass * mass), stat), 0, 100 * TF,
                          epsabs=0, epsrel=1e-13, limit=200)
    return g / (2 * np.pi ** 2) * v


def check_particle_number(plant=0):
    rng = np.random.default_rng(3)
    for stat in (-1, 1):
        for _ in range(3):
            tau, eta0 = rng.uniform(0.8, 3.0), rng.uniform(-1, 1)
            u = rng.uniform(-0.6, 0.6, 3)
            dS = rng.normal(size=4) * np.array([1.0, 0.5, 0.5, 0.5 * tau])
            r = _element(tau, eta0, dS, u)
            Y, wY, pT, wpT, phi, wphi = _grid(eta0)
            spec = oracle.cooper_frye(r[None], Y, pT, phi, M_PI, 1.0, stat, TF, viscous=False, plant=plant)
            N = _integrate(spec, wY, pT, wpT, wphi)
            udS = r[8] * dS[0] + u[0] * dS[1] + u[1] * dS[2] + u[2] / tau * dS[3]
            want = _density(stat) / HBARC ** 3 * udS
            assert abs(N - want) <= 1e-8 * abs(want) + 1e-12, (N, want)


def test_momentum_integral_is_the_thermal_density_times_u_dsigma():
    check_particle_number()


def _moment(k, stat, with_E=False):
    g = lambda p: p ** k * _f(np.sqrt(p * p + M_PI ** 2), stat) * (1 - stat * _f(np.sqrt(p * p + M_PI ** 2), stat)) \
        * (np.sqrt(p * p + M_PI ** 2) if with_E else 1.0)
    v, _ = integrate.quad(g, 0, 100 * TF, epsabs=0, epsrel=1e-13, limit=200)
    return v


def test_shear_moments_of_an_element_at_rest():
    """Only pi~^{xy}, pi~^{eta eta} or pi~^{tau x} nonzero on a tau = const
    element at rest at eta_s = 0: the p^x p^y, p_z^2 and p^x moments of the
    spectrum against one-dimensional integrals (rest-frame isotropy)."""
    V, ePf, stat = 2.0, 0.31, -1
    Y, wY, pT, wpT, phi, wphi = _grid(0.0)
    mT = np.sqrt(pT ** 2 + M_PI ** 2)
    px = (pT[:, None] * np.cos(phi)[None, :])[None]
    py = (pT[:, None] * np.sin(phi)[None, :])[None]
    pz = (np.sinh(Y)[:, None] * mT[None, :])[:, :, None]
    c = NORM * V / (TF ** 2 * ePf)
    a = 0.05
    pi = np.zeros(10)
    pi[5] = a
    spec = oracle.cooper_frye(_element(1.0, 0.0, [V, 0, 0, 0], [0, 0, 0], pi)[None], Y, pT, phi, M_PI, 1.0, stat,
                              TF, ePf)
    got = _integrate(spec, wY, pT, wpT, wphi, px * py)
    want = c * a * 4 * np.pi / 15 * _moment(6, stat)
    assert abs(got / want - 1) < 1e-8, (got, want)
    pi = np.zeros(10)
    pi[9] = a
    spec = oracle.cooper_frye(_element(1.0, 0.0, [V, 0, 0, 0], [0, 0, 0], pi)[None], Y, pT, phi, M_PI, 1.0, stat,
                              TF, ePf)
    got = _integrate(spec, wY, pT, wpT, wphi, pz * pz)
    iso, _ = integrate.quad(lambda p: p ** 4 * _f(np.sqrt(p * p + M_PI ** 2), stat), 0, 100 * TF, epsabs=0,
                            epsrel=1e-13, limit=200)
    want = NORM * V * 4 * np.pi / 3 * iso + c * a / 2 * 4 * np.pi / 5 * _moment(6, stat)
    assert abs(got / want - 1) < 1e-8, (got, want)
    pi = np.zeros(10)
    pi[1] = a
    spec = oracle.cooper_frye(_element(1.0, 0.0, [V, 0, 0, 0], [0, 0, 0], pi)[None], Y, pT, phi, M_PI, 1.0, stat,
                              TF, ePf)
    got = _integrate(spec, wY, pT, wpT, wphi, px)
    want = -c * a * 4 * np.pi / 3 * _moment(4, stat, with_E=True)
    assert abs(got / want - 1) < 1e-8, (got, want)


def test_bad_arguments_are_rejected():
    r = _element(1.0, 0.0, [1, 0, 0, 0], [0, 0, 0])[None]
    with pytest.raises(ValueError):
        oracle.cooper_frye(r, [0.0], [0.5], [0.0], M_PI, 1.0, -1, 0.0)
    with pytest.raises(ValueError):
        oracle.cooper_frye(r, [0.0], [0.5], [0.0], M_PI, 1.0, -1, TF, ePf=0.0, viscous=True)
