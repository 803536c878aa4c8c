"""Pins for the oracle's bulk pressure (reading R20; Eqs. Pi, Pitilde with
tau_Pi = 5 zeta/(T s)), against solutions the mathematics fixes.

  * Bjorken flow with shear and bulk: with u = (1,0,0,0), theta = 1/tau and
    u.nabla Pi = d_tau Pi, Eq. (Pi) and Eq. (bjorken) reduce to three ODEs.
  * A small sound wave in a static Cartesian box: linearising
    nabla_mu T^{mu nu} = 0 with T^{xx} = P + Pi + pi^{xx} and the relaxation
    equations of Pi and pi^{xx} gives a 4 x 4 linear system per Fourier mode,
    solved exactly by a matrix exponential.
  * The decomposition of Eq. (Tmn): after steps of a flowing event, the
    stored T~^{tau mu} equals (eps + P_t) u~^tau u~^mu - P_t g~^{tau mu}
    + pi~^{tau mu} of the stored primitives, P_t = max(P + Pi, 0) (what the
    root solve must invert).
  * Energy-momentum conservation in a periodic box, and zeta/s = 0 leaving
    every bit of the shear-only run unchanged.

Each ``check_*`` raises AssertionError when its pin fails; the planted-mistake
meta-test reuses them with deliberately broken oracle builds.
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.linalg import expm

import oracle
from conftest import assert_regulator_inactive
from paper_1802_04449_gb300 import inputs as I

HBARC = 0.1973269804


def _coeffs(e, eta_over_s, zeta_over_s):
    """(eta_v, tau_pi, zeta, tau_Pi) of the conformal gas at eps = e."""
    w = 4.0 * e / 3.0
    T = float(I.conformal_T(e))
    eta_v = eta_over_s * w * HBARC / T
    zeta = zeta_over_s * w * HBARC / T
    return eta_v, 5 * eta_v / w, zeta, 5 * zeta / w


# ------------------------------------------------------------ Bjorken
def bjorken_bulk_run(dtau, eta_over_s=0.08, zeta_over_s=0.12, tau0=0.6, tau1=1.6, e0=30.0, plant=0):
    """With phi = -tau^2 pi^{eta eta}:
      d eps/d tau = -(eps + P + Pi - phi)/tau,
      d phi/d tau = -(phi - 4 eta_v/(3 tau))/tau_pi - (4/3) phi/tau,
      d Pi/d tau  = -(Pi + zeta/tau)/tau_Pi - (4/3) Pi/tau."""
    o = oracle.Oracle(4, 4, 4, 0.3, 0.3, 0.3, tau0, dtau, eta_over_s=eta_over_s, zeta_over_s=zeta_over_s,
                      periodic=True, plant=plant)
    e = np.full((4, 4, 4), e0)
    z = np.zeros_like(e)
    o.set_initial(e, z, z, z)
    o.step(int(round((tau1 - tau0) / dtau)))
    f = o.fields()
    t = o.stats()["tau"]

    def rhs(tt, y):
        e, phi, Pi = y
        eta_v, tau_pi, zeta, tau_Pi = _coeffs(e, eta_over_s, zeta_over_s)
        return [-(e + e / 3 + Pi - phi) / tt,
                -(phi - 4 * eta_v / (3 * tt)) / tau_pi - (4.0 / 3.0) * phi / tt,
                -(Pi + zeta / tt) / tau_Pi - (4.0 / 3.0) * Pi / tt]

    s = solve_ivp(rhs, (tau0, t), [e0, 0.0, 0.0], method="DOP853", rtol=1e-12, atol=1e-14)
    return f, s.y[:, -1]


def check_bjorken_bulk(plant=0):
    errs = []
    for dtau in (0.02, 0.01):
        f, (e_ex, phi_ex, Pi_ex) = bjorken_bulk_run(dtau, plant=plant)
        if plant == 0:
            assert_regulator_inactive(f, f["eps"] / 3, f["Pi"])
        for k in ("eps", "Pi", "piee"):
            assert np.ptp(f[k]) == 0.0          # uniform stays exactly uniform
        assert Pi_ex < 0                        # expansion lowers the pressure
        errs.append((f["eps"][0, 0, 0] / e_ex - 1, -f["piee"][0, 0, 0] / phi_ex - 1, f["Pi"][0, 0, 0] / Pi_ex - 1))
    (e1, p1, b1), (e2, p2, b2) = errs
    assert abs(e1) < 1e-3 and abs(p1) < 1e-2 and abs(b1) < 1e-2, errs
    assert 3.4 < e1 / e2 < 4.6 and 3.4 < b1 / b2 < 4.6, errs   # second order in h (Heun)


def test_bjorken_bulk_ode():
    check_bjorken_bulk()


# ----------------------------------------------- linearised sound wave
def sound_wave_err(nx, plant=0, amp=1e-4, L=4.0, t1=2.0, e0=10.0, eta_over_s=0.16, zeta_over_s=0.1):
    """eps = e0 (1 + amp cos kx), u = 0 at t = 0 in a static Cartesian box.
    Per mode, with eps = e0 + A cos kx, u^x = B sin kx, pi^{xx} = C cos kx,
    Pi = D cos kx, w = 4 e0/3:
      A' = -w k B,   w B' = k (A/3 + C + D),
      C' = -(C + (4/3) eta_v k B)/tau_pi,   D' = -(D + zeta k B)/tau_Pi."""
    dx = L / nx
    k = 2 * np.pi / L
    x = (np.arange(nx) + 0.5) * dx
    dt = 0.2 * dx
    sh = (nx, 1, 1)
    o = oracle.Oracle(nx, 1, 1, dx, 1.0, 1.0, 0.0, dt, eta_over_s=eta_over_s, zeta_over_s=zeta_over_s,
                      cartesian=True, periodic=True, plant=plant)
    z = np.zeros(sh)
    o.set_initial((e0 * (1 + amp * np.cos(k * x))).reshape(sh), z, z, z)
    o.step(int(round(t1 / dt)))
    if plant == 0:
        f = o.fields()
        assert_regulator_inactive(f, f["eps"] / 3, f["Pi"])
    t = o.stats()["tau"]
    c, s = np.cos(k * x), np.sin(k * x)
    got = np.array([2 * np.mean(o.get("eps")[:, 0, 0] * c), 2 * np.mean(o.get("ux")[:, 0, 0] * s),
                    2 * np.mean(o.get("pixx")[:, 0, 0] * c), 2 * np.mean(o.get("Pi")[:, 0, 0] * c)])
    w = 4 * e0 / 3
    eta_v, tau_pi, zeta, tau_Pi = _coeffs(e0, eta_over_s, zeta_over_s)
    M = np.array([[0, -w * k, 0, 0],
                  [k / (3 * w), 0, k / w, k / w],
                  [0, -(4 / 3) * eta_v * k / tau_pi, -1 / tau_pi, 0],
                  [0, -zeta * k / tau_Pi, 0, -1 / tau_Pi]])
    ex = expm(M * t) @ np.array([amp * e0, 0, 0, 0])
    scale = np.array([amp * e0, amp, amp * e0, amp * e0])
    return np.abs(got - ex) / scale, ex / scale


def check_bulk_sound_wave(plant=0):
    r1, _ = sound_wave_err(32, plant=plant)
    r2, ex = sound_wave_err(64, plant=plant)
    assert abs(ex[3]) > 0.02 and abs(ex[2]) > 0.02   # both viscous modes are excited
    assert np.all(r2 < 2e-3), (r1, r2)
    assert np.all(r1 / r2 > 2.5), (r1, r2)


def test_sound_wave_with_shear_and_bulk():
    check_bulk_sound_wave()


# ------------------------------------------------------ decomposition
def decomposition_err(plant=0, zeta_over_s=0.2, nsteps=12):
    case = I.hotspot_event(nx=13, ny=11, neta=9, n_spots=12, seed=6)
    o = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                      case.eta_over_s, case.eos, case.cartesian, case.periodic, plant=plant,
                      zeta_over_s=zeta_over_s)
    o.set_initial(case.eps, case.ux, case.uy, case.ueta)
    o.step(nsteps)
    f = o.fields()
    tau = o.stats()["tau"]
    e = f["eps"]
    P = np.maximum(np.vectorize(lambda x: o.eos(x)[0])(e) + f["Pi"], 0.0)
    u = [f["ux"], f["uy"], f["ueta"]]
    ut = np.sqrt(1 + u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    w = e + P
    want = [w * ut * ut - P + f["pitt"], w * ut * u[0] + f["pitx"], w * ut * u[1] + f["pity"],
            w * ut * u[2] + f["pite"]]
    got = [f[k] / tau for k in ("Ttt", "Ttx", "Tty", "Tte")]   # T~^{tau mu} = tau T^{tau mu}
    scale = np.abs(got[0]).max()
    live = e > 0
    Pi_rel = np.abs(f["Pi"][live] / P[live]).max()
    return max(np.abs(g - h_)[live].max() for g, h_ in zip(got, want)) / scale, Pi_rel


def check_decomposition(plant=0):
    err, Pi_rel = decomposition_err(plant=plant)
    assert Pi_rel > 0.02                # the bulk pressure is not negligible
    assert err < 1e-12, err


def test_decomposition_of_T_with_bulk():
    check_decomposition()


# ------------------------------------------------- root solve with Pi
def test_root_solve_with_bulk_pressure_is_the_unique_root():
    """For random (eps, v, Pi) with |Pi| <= P(eps) and the table EOS, build
    E = (eps + P_t) gamma^2 - P_t and M = (eps + P_t) gamma^2 v with
    P_t = max(P(eps) + Pi, 0): the solve returns (eps, v).  Where the total
    pressure floor binds nearby, f(v) = v - M/(E + P_t(E - M v)) still has a
    single sign change on [0, M/E] (brute force on 4001 points)."""
    eos = I.crossover_eos()
    o = oracle.Oracle(2, 2, 2, 0.3, 0.3, 0.3, 0.6, 0.01, eta_over_s=0.1, zeta_over_s=0.1, eos=eos)
    rng = np.random.default_rng(4)
    Pt = lambda x, Pi: max(o.eos(x)[0] + Pi, 0.0)
    for _ in range(150):
        e = 10 ** rng.uniform(-2.5, 1.5)
        v = rng.uniform(0, 0.95)
        Pi = rng.uniform(-1.05, 1.0) * o.eos(e)[0]   # a little beyond -P: the floor binds
        w = e + Pt(e, Pi)
        g2 = 1 / (1 - v * v)
        E, M = w * g2 - Pt(e, Pi), w * g2 * v
        out = o.prim_bulk(E, M, 0.0, 0.0, Pi)
        assert out[5] > 0
        assert abs(out[0] / e - 1) < 1e-11 and abs(out[2] / out[1] - v) < 1e-11, (e, v, Pi, out)
        vs = np.linspace(0, M / E, 4001)
        f = np.array([x - M / (E + Pt(E - M * x, Pi)) for x in vs])
        assert np.sum(np.diff(np.sign(f)) != 0) == 1


# ------------------------------------------------ conservation, limits
def test_periodic_box_conserves_energy_momentum_with_bulk():
    rng = np.random.default_rng(9)
    nx, ny, ne = 12, 10, 8
    eps, ux, uy, ue = I.random_smooth_box(rng, nx, ny, ne)
    o = oracle.Oracle(nx, ny, ne, 0.3, 0.3, 0.3, 0.0, 0.02, eta_over_s=0.1, zeta_over_s=0.2, cartesian=True,
                      periodic=True)
    o.set_initial(eps, ux, uy, ue)
    q0 = [o.get(k).sum() for k in ("Ttt", "Ttx", "Tty", "Tte")]
    o.step(40)
    q1 = [o.get(k).sum() for k in ("Ttt", "Ttx", "Tty", "Tte")]
    assert np.abs(o.get("Pi")).max() > 1e-3 * eps.max()   # bulk pressure has built up
    for a, b in zip(q0, q1):
        assert abs(b - a) <= 1e-12 * abs(q0[0])


def test_zero_zeta_leaves_shear_run_unchanged():
    case = I.hotspot_event(nx=11, ny=9, neta=7, n_spots=10, seed=2)
    runs = []
    for zs in (None, 0.0):
        kw = {} if zs is None else {"zeta_over_s": zs}
        o = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                          case.eta_over_s, case.eos, case.cartesian, case.periodic, **kw)
        o.set_initial(case.eps, case.ux, case.uy, case.ueta)
        o.step(8)
        runs.append(o.fields())
        assert np.all(runs[-1]["Pi"] == 0)
    for k in runs[0]:
        np.testing.assert_array_equal(runs[0][k], runs[1][k])


def test_bulk_needs_shear_and_a_nonnegative_ratio():
    with pytest.raises(ValueError):
        oracle.Oracle(4, 4, 4, 0.3, 0.3, 0.3, 0.6, 0.01, eta_over_s=0.0, zeta_over_s=0.1)
    with pytest.raises(ValueError):
        oracle.Oracle(4, 4, 4, 0.3, 0.3, 0.3, 0.6, 0.01, eta_over_s=0.1, zeta_over_s=-0.1)
