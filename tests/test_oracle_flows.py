"""Pins for the oracle's full Heun step against solutions the paper and the
mathematics fix (Sec. 5 tests of the paper, plus conservation and a
linearised longitudinal sound wave).

Each ``check_*`` function raises AssertionError when the pin fails; the
planted-mistake meta-test reuses them with deliberately broken oracle builds.
"""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle
from conftest import assert_regulator_inactive
from paper_1802_04449_gb300 import inputs as I

HBARC = 0.1973269804


def uniform(n, e0):
    e = np.full((n, n, n), e0)
    z = np.zeros_like(e)
    return e, z, z, z


# ---------------------------------------------------------------- Bjorken
def bjorken_ideal_err(dtau, eos=None, tau0=0.6, tau1=1.6, e0=30.0, plant=0):
    o = oracle.Oracle(4, 4, 4, 0.3, 0.3, 0.3, tau0, dtau, eos=eos, periodic=True, plant=plant)
    o.set_initial(*uniform(4, e0))
    o.step(int(round((tau1 - tau0) / dtau)))
    e = o.get("eps")
    assert np.ptp(e) == 0.0  # uniform stays exactly uniform
    t = o.stats()["tau"]
    if eos is None:
        exact = e0 * (tau0 / t) ** (4.0 / 3.0)   # ideal conformal Bjorken
    else:
        lne = eos["lne0"] + eos["dlne"] * np.arange(len(eos["P"]))
        P = lambda x: np.interp(np.log(x), lne, eos["P"])
        # Eq. (bjorken) with pi = 0: d eps/d tau = -(eps + P)/tau
        s = solve_ivp(lambda tt, y: [-(y[0] + P(y[0])) / tt], (tau0, t), [e0], method="DOP853",
                      rtol=1e-12, atol=1e-14)
        exact = s.y[0, -1]
    return e[0, 0, 0] / exact - 1.0


def check_bjorken_ideal(plant=0, eos=None):
    e1 = bjorken_ideal_err(0.02, eos, plant=plant)
    e2 = bjorken_ideal_err(0.01, eos, plant=plant)
    assert abs(e1) < 5e-4
    assert 3.6 < e1 / e2 < 4.4, (e1, e2)   # second order in h (Heun)


def test_bjorken_ideal_conformal():
    check_bjorken_ideal()


def test_bjorken_ideal_table_eos():
    check_bjorken_ideal(eos=I.crossover_eos())


def bjorken_viscous_run(dtau, eta_over_s=0.16, tau0=0.6, tau1=1.6, e0=30.0, plant=0):
    """Viscous Bjorken flow, conformal EOS.  With u = (1,0,0,0), theta = 1/tau,
    tau^2 sigma^{eta eta} = -4/(3 tau), and u.nabla pi^{eta eta} =
    d_tau pi^{eta eta} + 2 pi^{eta eta}/tau, the Israel-Stewart equation for
    phi = -tau^2 pi^{eta eta} and Eq. (bjorken) give
      d eps/d tau = -(eps + P - phi)/tau,
      d phi/d tau = -(phi - 4 eta_v/(3 tau))/tau_pi - (4/3) phi/tau,
    eta_v = (eta/s)(eps+P) hbar c/T, tau_pi = 5 eta_v/(eps+P)."""
    o = oracle.Oracle(4, 4, 4, 0.3, 0.3, 0.3, tau0, dtau, eta_over_s=eta_over_s, periodic=True,
                      plant=plant)
    o.set_initial(*uniform(4, e0))
    o.step(int(round((tau1 - tau0) / dtau)))
    f = o.fields()
    t = o.stats()["tau"]

    def rhs(tt, yv):
        e, phi = yv
        P = e / 3
        T = float(I.conformal_T(e))
        eta_v = eta_over_s * (e + P) * HBARC / T
        tau_pi = 5 * eta_v / (e + P)
        return [-(e + P - phi) / tt, -(phi - 4 * eta_v / (3 * tt)) / tau_pi - (4.0 / 3.0) * phi / tt]

    s = solve_ivp(rhs, (tau0, t), [e0, 0.0], method="DOP853", rtol=1e-12, atol=1e-14)
    return f, s.y[0, -1], s.y[1, -1]


def check_bjorken_viscous(plant=0):
    errs = []
    for dtau in (0.02, 0.01):
        f, e_ex, phi_ex = bjorken_viscous_run(dtau, plant=plant)
        if plant == 0:
            assert_regulator_inactive(f, f["eps"] / 3)
        phi = -f["piee"][0, 0, 0]
        errs.append((f["eps"][0, 0, 0] / e_ex - 1, phi / phi_ex - 1))
        # symmetry and tracelessness of Bjorken flow: pi^xx = pi^yy = phi/2, pi^tt = 0
        np.testing.assert_allclose(f["pixx"], phi / 2, rtol=1e-12)
        np.testing.assert_allclose(f["piyy"], phi / 2, rtol=1e-12)
        assert np.all(f["pitt"] == 0)
    (e1, p1), (e2, p2) = errs
    assert abs(e1) < 1e-3 and abs(p1) < 1e-2, errs
    assert 3.4 < e1 / e2 < 4.6 and 3.4 < p1 / p2 < 4.6, errs


def test_bjorken_viscous_ode():
    check_bjorken_viscous()


# ---------------------------------------------------------------- Gubser
def gubser_err(dx, tau1=1.6, plant=0):
    half = 4.8
    nx = int(round(2 * half / dx)) + 1
    c = I.gubser_case(dx=dx, nx=nx, neta=1, deta=0.3, dtau=dx / 10, tau1=tau1)
    o = oracle.Oracle(c.nx, c.ny, 1, c.dx, c.dy, c.deta, c.tau0, c.dtau, plant=plant)
    o.set_initial(c.eps, c.ux, c.uy, c.ueta)
    o.step(c.nsteps)
    x = I.cell_coords(c.nx, c.dx)
    ea, uxa, _ = I.gubser_ideal(o.stats()["tau"], x, x)
    X, Y = np.meshgrid(x, x, indexing="ij")
    m = X ** 2 + Y ** 2 <= 2.5 ** 2
    eo, uxo = o.get("eps")[:, :, 0], o.get("ux")[:, :, 0]
    return (np.abs(eo - ea)[m].sum() / np.abs(ea[m]).sum(),
            np.abs(uxo - uxa)[m].sum() / np.abs(uxa[m]).sum())


def check_gubser(plant=0):
    (e1, u1), (e2, u2), (e3, u3) = (gubser_err(dx, plant=plant) for dx in (0.3, 0.15, 0.075))
    info = (e1, e2, e3, u1, u2, u3)
    assert e3 < 0.015 and u3 < 0.012, info
    # minmod clips the moving ring: the observed order rises towards 2 with resolution
    assert e1 > e2 > e3 and u1 > u2 > u3, info
    assert e2 / e3 > 2.2 and u2 / u3 > 2.8, info


def test_gubser_ideal_convergence():
    """Ideal conformal Gubser flow (Sec. 5, lambda_1 -> infinity): L1 error in
    eps and u~^x for r <= 2.5 fm falls under refinement (dx 0.3, 0.15, 0.075)."""
    check_gubser()


# ---------------------------------------------------------------- Riemann
def riemann_err(dx, plant=0):
    nx = int(round(12 / dx)) + 1
    x, e = I.riemann_1d(nx, dx, 10.0)
    sh = (nx, 1, 1)
    z = np.zeros(sh)
    dt = 0.25 * dx
    o = oracle.Oracle(nx, 1, 1, dx, 1, 1, tau0=0.0, dtau=dt, cartesian=True, plant=plant)
    o.set_initial(e.reshape(sh), z, z, z)
    o.step(int(round(4.0 / dt)))
    t = o.stats()["tau"]
    ea = I.riemann_exact(x / t, 10.0, 1 / math.sqrt(3))
    m = np.abs(x / t) < 0.9
    return np.abs(o.get("eps")[:, 0, 0] - ea)[m].sum() * dx


def test_riemann_rarefaction_convergence():
    """Cartesian mode (Christoffel terms off), step IC of Eq. (riemann):
    L1 error against the rarefaction closed form halves with dx."""
    e1, e2 = riemann_err(0.1), riemann_err(0.05)
    assert e2 < 0.7 and 1.7 < e1 / e2 < 2.5, (e1, e2)


# -------------------------------------------- longitudinal sound wave (Milne)
def eta_wave_err(ne, plant=0, amp=1e-4, L=2.0, tau0=1.0, tau1=2.0, e0=10.0):
    """Small wave e = e0(1 + d cos k eta), u~^eta = w sin k eta on ideal
    conformal Bjorken flow.  Linearising nabla_mu T^{mu nu} = 0 in Milne
    coordinates around eps_0(tau) ~ tau^{-4/3}, u = (1,0,0,0) gives
      d' = -(4/3) k w / tau,    w' = k d/(4 tau) - (2/3) w/tau."""
    deta = L / ne
    k = 2 * np.pi / L
    eta = (np.arange(ne) + 0.5) * deta
    sh = (1, 1, ne)
    dt = 0.1 * tau0 * deta
    o = oracle.Oracle(1, 1, ne, 1, 1, deta, tau0=tau0, dtau=dt, periodic=True, plant=plant)
    z = np.zeros(sh)
    o.set_initial((e0 * (1 + amp * np.cos(k * eta))).reshape(sh), z, z, (amp * np.sin(k * eta)).reshape(sh))
    o.step(int(round((tau1 - tau0) / dt)))
    t = o.stats()["tau"]
    eo, uo = o.get("eps")[0, 0], o.get("ueta")[0, 0]
    d = 2 * np.mean((eo / eo.mean() - 1) * np.cos(k * eta))
    w = 2 * np.mean(uo * np.sin(k * eta))
    s = solve_ivp(lambda tt, y: [-(4 / 3) * k * y[1] / tt, k * y[0] / (4 * tt) - (2 / 3) * y[1] / tt],
                  (tau0, t), [amp, amp], method="DOP853", rtol=1e-12, atol=1e-18)
    mean_err = eo.mean() / (e0 * (tau0 / t) ** (4 / 3)) - 1
    return abs(d - s.y[0, -1]) / amp, abs(w - s.y[1, -1]) / amp, abs(mean_err)


def check_eta_wave(plant=0):
    d1, w1, m1 = eta_wave_err(32, plant=plant)
    d2, w2, m2 = eta_wave_err(64, plant=plant)
    assert d2 < 4e-3 and w2 < 4e-3 and m2 < 1e-6, (d1, d2, w1, w2, m2)
    assert d1 / d2 > 3.0 and w1 / w2 > 3.0, (d1, d2, w1, w2)


def test_eta_wave_linearised_milne():
    check_eta_wave()


# --------------------------------------------------------- conservation
def test_periodic_box_conserves_energy_momentum():
    """Cartesian mode, periodic box, viscous: sum over cells of T^{t mu}
    changes only by rounding (KT flux differences telescope)."""
    rng = np.random.default_rng(1)
    n = 10
    e, ux, uy, ue = I.random_smooth_box(rng, n, n, n)
    o = oracle.Oracle(n, n, n, 0.2, 0.2, 0.2, tau0=1.0, dtau=0.02, eta_over_s=0.16, cartesian=True,
                      periodic=True)
    o.set_initial(e, ux, uy, ue)
    keys = ("Ttt", "Ttx", "Tty", "Tte")
    T0 = np.array([o.get(k).sum() for k in keys])
    o.step(150)
    T1 = np.array([o.get(k).sum() for k in keys])
    assert np.all(np.abs(T1 - T0) <= 1e-13 * T0[0])
    assert np.abs(o.get("pixx")).max() > 1e-3   # the viscous part is active


# ------------------------------------------------- transversality drift
def transversality_drift(ne, plant=0, L=2.0, tau1=1.4):
    deta = L / ne
    k = 2 * np.pi / L
    eta = (np.arange(ne) + 0.5) * deta
    sh = (1, 1, ne)
    dt = 0.05 * deta
    o = oracle.Oracle(1, 1, ne, 1, 1, deta, tau0=1.0, dtau=dt, eta_over_s=0.16, periodic=True,
                      plant=plant)
    z = np.zeros(sh)
    o.set_initial((10 * (1 + 0.3 * np.cos(k * eta))).reshape(sh), z, z, (0.3 * np.sin(k * eta)).reshape(sh))
    o.step(int(round((tau1 - 1.0) / dt)))
    f = o.fields()
    ut = np.sqrt(1 + f["ueta"] ** 2)
    scale = max(np.abs(f["pi" + a]).max() for a in ("tt", "te", "ee", "xx", "yy"))
    # u~_mu pi~^{mu nu} with g~ = diag(1,-1,-1,-1): nu = tau and nu = eta
    t_tau = ut * f["pitt"] - f["ueta"] * f["pite"]
    t_eta = ut * f["pite"] - f["ueta"] * f["piee"]
    trace = f["pitt"] - f["pixx"] - f["piyy"] - f["piee"]
    return max(np.abs(t_tau).max(), np.abs(t_eta).max()) / scale, np.abs(trace).max() / scale


def check_transversality(plant=0):
    """Israel-Stewart preserves u_mu pi^{mu nu} = 0 and pi^mu_mu = 0; the
    discrete drift must shrink under refinement.  A wrong I^{mu nu} sign or a
    wrong Christoffel correction leaves an O(1) drift (Sec. 2, Eq. Ipi)."""
    (t1, r1), (t2, r2) = transversality_drift(16, plant), transversality_drift(64, plant)
    assert t2 < 4e-3 and t2 < t1 / 3.0, (t1, t2)
    assert r2 < 2e-3 and r2 < r1 / 1.8, (r1, r2)


def test_transversality_and_trace_drift():
    check_transversality()


# --------------------------------------------------------- determinism
def test_thread_count_does_not_change_bits():
    case = I.hotspot_event(nx=17, ny=15, neta=7, n_spots=40, seed=5)
    outs = []
    for nt in (1, 4):
        oracle.set_threads(nt)
        o = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0,
                          case.dtau, case.eta_over_s, case.eos)
        o.set_initial(case.eps, case.ux, case.uy, case.ueta)
        o.step(3)
        outs.append(o.fields())
    oracle.set_threads(0)
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k


# ------------------------------------------------------- shear regulator
def test_shear_regulator_caps_oversized_pi():
    check_regulator_cap()


def check_regulator_cap(plant=0):
    """Reading R18: after a stage, |pi_{mu nu} pi^{mu nu}| <= eps^2 + 3 P^2
    (eps, P of the stage input).  Uniform Bjorken cells with an initial
    pi~^{xx} = pi~^{yy} = -pi~^{ee}/2 ten times eps: the first stage scales pi
    onto the bound, so the evolved pi is far below the unregulated value."""
    n, e0 = 4, 10.0
    e = np.full((n, n, n), e0)
    z = np.zeros_like(e)
    pi = np.zeros((10, n, n, n))
    pi[4] = pi[7] = 10 * e0
    pi[9] = -20 * e0
    o = oracle.Oracle(n, n, n, 0.3, 0.3, 0.3, 1.0, 0.01, eta_over_s=0.16, periodic=True, plant=plant)
    o.set_initial(e, z, z, z, pi)
    o.step(1)
    f = o.fields()
    P = f["eps"] / 3.0
    pp = f["pixx"] ** 2 + f["piyy"] ** 2 + f["piee"] ** 2
    # the second stage caps pi with the stage-1 eps' (the large negative
    # pi~^{ee} raised eps); the result sits at the bound of an eps between
    # the initial and the final value, far below the unregulated ~200
    bound = lambda x: np.sqrt(x ** 2 + 3 * (x / 3) ** 2)
    assert np.all(np.sqrt(pp) <= 1.05 * bound(1.1 * f["eps"]))
    assert np.all(np.sqrt(pp) >= 0.95 * bound(e0))
    assert np.all(np.isfinite(f["eps"])) and np.all(f["eps"] > 0)


def test_shear_regulator_cap_is_exact_in_a_static_box():
    check_regulator_cap_exact()


def check_regulator_cap_exact(plant=0):
    """Reading R18's cap in a static, uniform Cartesian box: no gradient, so
    T~ and eps stay put (pi~^{tau mu} = 0 at rest) and only the relaxation
    acts on pi.  With pi~^{xx} = pi~^{yy} = -pi~^{zz}/2 ten times eps, both
    stages exceed the bound, so after the step |pi_{mu nu} pi^{mu nu}| sits
    exactly on eps^2 + 3 P^2 of the (unchanged) eps, the conformal P = eps/3."""
    n, e0 = 2, 10.0
    e = np.full((n, n, n), e0)
    z = np.zeros_like(e)
    pi = np.zeros((10, n, n, n))
    pi[4] = pi[7] = 10 * e0
    pi[9] = -20 * e0
    o = oracle.Oracle(n, n, n, 0.3, 0.3, 0.3, 1.0, 0.01, eta_over_s=0.16, cartesian=True, periodic=True,
                      plant=plant)
    o.set_initial(e, z, z, z, pi)
    o.step(1)
    f = o.fields()
    np.testing.assert_allclose(f["eps"], e0, rtol=1e-14)
    pp = f["pixx"] ** 2 + f["piyy"] ** 2 + f["piee"] ** 2
    np.testing.assert_allclose(np.sqrt(pp), np.sqrt(e0 ** 2 + 3 * (e0 / 3) ** 2), rtol=1e-12)
    np.testing.assert_allclose(f["pixx"] / f["piee"], -0.5, rtol=1e-12)     # the cap scales, keeps the shape


def test_shear_regulator_ramp_static_box():
    check_regulator_ramp()


def check_regulator_ramp(plant=0):
    """Reading R18's ramp r(eps) = clamp(eps/1e-3 - 1, 0, 1).  In a static,
    uniform Cartesian box every gradient vanishes, T~ and eps stay put, and
    the IS equation reduces to d pi/dt = -pi/tau_pi.  One Heun step with the
    regulator after each stage then gives, with k = 1 - h/tau_pi,
    pi' = r k pi and pi^{n+1} = r (pi + pi' k)/2 = r (1 + r k^2) pi / 2.
    Cells at eps = 0.9e-3, 1.4e-3 and 2.5e-3 span the three branches; pi~^{xy}
    is small, so the cap of R18 stays inactive."""
    n, h, a = 2, 0.01, 1e-7
    for e0, r in ((0.9e-3, 0.0), (1.4e-3, 0.4), (2.5e-3, 1.0)):
        e = np.full((n, n, n), e0)
        z = np.zeros_like(e)
        pi = np.zeros((10, n, n, n))
        pi[5] = a
        o = oracle.Oracle(n, n, n, 0.3, 0.3, 0.3, 1.0, h, eta_over_s=0.16, cartesian=True, periodic=True,
                          plant=plant)
        o.set_initial(e, z, z, z, pi)
        o.step(1)
        f = o.fields()
        _, T, _ = o.eos(e0)
        k = 1.0 - h * T / (5 * 0.16 * HBARC)
        want = 0.5 * r * (1.0 + r * k * k) * a
        np.testing.assert_allclose(f["pixy"], want, rtol=1e-12, atol=1e-30)
        np.testing.assert_allclose(f["eps"], e0, rtol=1e-14)
        assert np.all(f["pitt"] == 0) and np.all(f["pixx"] == 0)
