"""Seeded synthetic inputs shared by the oracle and the CUDA path.

Nothing here is part of the hydro method: these functions only build initial
conditions and the equation-of-state table that both implementations receive
as inputs.  The paper's workloads (Trento / AMPT events, lattice and HRG EOS
tables) are not available; the generators below stand in for them with the
same shapes, scales and structure.

Units: lengths in fm, energy density in GeV/fm^3, temperature in GeV.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

HBARC = 0.1973269804  # GeV fm
DOF_CONF = 47.5       # degeneracy of the conformal u, d, s + gluon gas


def cell_coords(n: int, d: float) -> np.ndarray:
    """Cell centres x_i = (i - (n-1)/2) d."""
    return (np.arange(n) - (n - 1) / 2.0) * d


# --------------------------------------------------------------------------
# equation of state tables
# --------------------------------------------------------------------------
def conformal_T(eps):
    """Temperature of the conformal gas with eps = 3 g pi^2 T^4 / (90 (hbar c)^3)."""
    eps = np.asarray(eps, dtype=np.float64)
    return np.where(eps > 0, (30.0 * HBARC ** 3 * np.maximum(eps, 0) / (DOF_CONF * math.pi ** 2)) ** 0.25, 0.0)


def crossover_cs2(eps):
    """Synthetic crossover: c_s^2(eps) = 1/3 - 0.2 exp(-ln^2(eps/0.5)/2)."""
    eps = np.asarray(eps, dtype=np.float64)
    return 1.0 / 3.0 - 0.2 * np.exp(-0.5 * np.log(eps / 0.5) ** 2)


def crossover_eos_table(n: int = 4096, eps_lo: float = 1e-7, eps_hi: float = 1e4, oversample: int = 64):
    """Thermodynamically consistent stand-in for a lattice/HRG crossover EOS.

    P = int_0^eps c_s^2, ln s = int d eps/(eps + P) + const, T = (eps + P)/s,
    with the constant fixed so that T matches the conformal gas at eps = 1e3.
    Returns nodes uniform in ln(eps): dict(lne0, dlne, P, T, cs2, eps).
    """
    lne0, lne1 = math.log(eps_lo), math.log(eps_hi)
    m = (n - 1) * oversample + 1
    x = np.linspace(lne0, lne1, m)
    e = np.exp(x)
    cs2 = crossover_cs2(e)
    # P(eps_lo) from c_s^2 = 1/3 below the first node (the Gaussian term is
    # ~exp(-118) there), then cumulative Simpson-like trapezoid in ln(eps).
    integrand = cs2 * e
    P = np.empty(m)
    P[0] = eps_lo / 3.0
    P[1:] = P[0] + np.cumsum(0.5 * (integrand[1:] + integrand[:-1]) * np.diff(x))
    g = e / (e + P)
    lns = np.empty(m)
    lns[0] = 0.0
    lns[1:] = np.cumsum(0.5 * (g[1:] + g[:-1]) * np.diff(x))
    Tref = float(conformal_T(1e3))
    lns_ref = np.interp(math.log(1e3), x, lns)
    P_ref = np.interp(math.log(1e3), x, P)
    # T = (eps + P)/s  ->  s_ref = (1e3 + P_ref)/Tref at eps = 1e3
    s = np.exp(lns - lns_ref) * (1e3 + P_ref) / Tref
    T = (e + P) / s
    sel = slice(0, m, oversample)
    dlne = (lne1 - lne0) / (n - 1)
    return {"lne0": lne0, "dlne": dlne, "P": P[sel].copy(), "T": T[sel].copy(),
            "cs2": cs2[sel].copy(), "eps": e[sel].copy()}


# --------------------------------------------------------------------------
# analytic-solution initial conditions
# --------------------------------------------------------------------------
def gubser_ideal(tau, x, y, q=1.0, eps_norm=10.0):
    """Ideal conformal Gubser flow (Sec. 5, Eqs. conformal, visc_gubser with
    lambda_1 -> infinity): eps = C (2q)^{8/3} tau^{-4/3} /
    [1 + 2 q^2 (tau^2 + r^2) + q^4 (tau^2 - r^2)^2]^{4/3}, outward
    v_perp = 2 q^2 tau r / (1 + q^2 tau^2 + q^2 r^2).  C is fixed so that
    eps(tau=1 fm, r=0) = eps_norm.  Returns eps, u~^x, u~^y."""
    def raw(t, r2):
        return (2 * q) ** (8.0 / 3.0) * t ** (-4.0 / 3.0) / (
            1 + 2 * q * q * (t * t + r2) + q ** 4 * (t * t - r2) ** 2) ** (4.0 / 3.0)
    C = eps_norm / raw(1.0, 0.0)
    X, Y = np.meshgrid(x, y, indexing="ij")
    r2 = X * X + Y * Y
    r = np.sqrt(r2)
    eps = C * raw(tau, r2)
    vr = 2 * q * q * tau * r / (1 + q * q * tau * tau + q * q * r2)
    gam = 1.0 / np.sqrt(1 - vr * vr)
    with np.errstate(invalid="ignore", divide="ignore"):
        cx = np.where(r > 0, X / r, 0.0)
        cy = np.where(r > 0, Y / r, 0.0)
    return eps, gam * vr * cx, gam * vr * cy


def gubser_viscous(tau, x, y, L=2.0, lambda1_hat=-10.0, eps_norm=10.0):
    """Second-order viscous Gubser flow (Sec. 5, Eqs. weyl_transform,
    conformal, visc_gubser_before_weyl, gubser_viscous): uniform in the
    de Sitter coordinates (rho, theta), eps_hat = C cosh(rho)^-(8/3 - 2/l1),
    pi_hat^{eta eta} = 2 eps_hat / l1, pi_hat^{theta theta} cosh^2 rho =
    pi_hat^{phi phi} cosh^2 rho sin^2 theta = -eps_hat / l1 (l1 = lambda1_hat),
    mapped back by the Weyl rescaling: eps = eps_hat / tau^4, outward
    v_perp = 2 tau r / (L^2 + tau^2 + r^2), pi_{mu nu} = tau^-2 (d xhat / d x)
    (d xhat / d x) pi_hat.  Holds when eta_hat lambda1_hat^2 = 3 tau_pi_hat.
    C is fixed so that eps(tau = 1 fm, r = 0) = eps_norm.
    Returns eps, u~^x, u~^y and pi~ (10, packed tt tx ty te xx xy xe yy ye ee)."""
    l1 = float(lambda1_hat)
    expo = 4.0 / 3.0 - 1.0 / l1          # cosh^2(rho) power: cosh(rho)^-(8/3 - 2/l1)

    def Qof(t, r2):                       # 4 L^2 tau^2 cosh^2 rho
        return L ** 4 + t ** 4 + r2 * r2 + 2 * L * L * t * t + 2 * L * L * r2 - 2 * t * t * r2

    def ehat(t, r2):
        return (Qof(t, r2) / (4 * L * L * t * t)) ** (-expo)

    C = eps_norm / (ehat(1.0, 0.0) / 1.0)
    X, Y = np.meshgrid(x, y, indexing="ij")
    r2 = X * X + Y * Y
    r = np.sqrt(r2)
    eh = C * ehat(tau, r2)
    eps = eh / tau ** 4
    S = L * L + tau * tau + r2
    vr = 2 * tau * r / S
    gam = 1.0 / np.sqrt(1 - vr * vr)
    with np.errstate(invalid="ignore", divide="ignore"):
        cx = np.where(r > 0, X / r, 0.0)
        cy = np.where(r > 0, Y / r, 0.0)
    Q = Qof(tau, r2)
    k = eh / l1
    p_tt = -4 * r2 * k / (tau ** 2 * Q)
    p_tr = -2 * r * S * k / (tau ** 3 * Q)          # pi^{tau r}
    p_rr = -S * S * k / (tau ** 4 * Q)
    p_pp = -k / tau ** 4                            # r^2 pi^{phi phi}
    pi = np.zeros((10,) + eps.shape)
    pi[0] = p_tt
    pi[1] = p_tr * cx
    pi[2] = p_tr * cy
    pi[4] = p_rr * cx * cx + p_pp * cy * cy
    pi[5] = (p_rr - p_pp) * cx * cy
    pi[7] = p_rr * cy * cy + p_pp * cx * cx
    pi[9] = 2 * k / tau ** 4                        # tau^2 pi^{eta eta}
    # at r = 0 the transverse block is isotropic
    pi[4] = np.where(r > 0, pi[4], p_pp)
    pi[7] = np.where(r > 0, pi[7], p_pp)
    return eps, gam * vr * cx, gam * vr * cy, pi


def gubser_viscous_case(dx=0.2, nx=41, neta=5, deta=0.2, dtau=0.01, tau0=1.0, tau1=1.5, L=2.0,
                        lambda1_hat=-10.0, eta_over_s=0.2):
    """Viscous Gubser flow on a Milne grid (conformal EOS, eta/s = 0.2,
    lambda1_hat = -10, tau_pi from eta_hat lambda1_hat^2 = 3 tau_pi_hat, i.e.
    tau_pi = (4 lambda1_hat^2 / 9) eta_v / (eps + P)), with the initial pi~
    and both coefficients in the case."""
    x = cell_coords(nx, dx)
    eps2, ux2, uy2, pi2 = gubser_viscous(tau0, x, x, L, lambda1_hat)
    rep = lambda a: np.repeat(a[..., None], neta, axis=-1)
    nsteps = int(round((tau1 - tau0) / dtau))
    return HydroCase("viscous Gubser flow", nx, nx, neta, dx, dx, deta, tau0, dtau, eta_over_s, None,
                     rep(eps2), rep(ux2), rep(uy2), np.zeros((nx, nx, neta)), nsteps,
                     pi0=rep(pi2), taupi_coef=4.0 * lambda1_hat ** 2 / 9.0, lambda1_hat=lambda1_hat)


def riemann_1d(nx, dx, eps0=10.0, t0=0.0):
    """Step initial condition along x (Sec. 5, Eq. riemann): eps0 for x <= 0,
    vacuum for x > 0, fluid at rest."""
    x = cell_coords(nx, dx)
    eps = np.where(x <= 1e-12, eps0, 0.0)
    return x, eps


def riemann_exact(zeta, eps0, cs):
    """Rarefaction solution of Eq. (riemann) as a function of zeta = x/t."""
    zeta = np.asarray(zeta, dtype=np.float64)
    out = np.zeros_like(zeta)
    left = zeta <= -cs
    mid = (zeta > -cs) & (zeta < 1.0)
    out[left] = eps0
    z = zeta[mid]
    out[mid] = eps0 * (((1 - cs) / (1 + cs)) * (1 - z) / (1 + z)) ** ((1 + cs * cs) / (2 * cs))
    return out


# --------------------------------------------------------------------------
# hot-spot event initial conditions (stand-in for Trento / AMPT events)
# --------------------------------------------------------------------------
WS_R, WS_A, WS_RHO0 = 6.62, 0.546, 0.17  # Pb Woods-Saxon


def _thickness_table(R=WS_R, a=WS_A, rho0=WS_RHO0, rmax=20.0, nr=801, nz=1601):
    r = np.linspace(0.0, rmax, nr)
    z = np.linspace(-rmax, rmax, nz)
    rr = np.sqrt(r[:, None] ** 2 + z[None, :] ** 2)
    rho = rho0 / (1.0 + np.exp((rr - R) / a))
    Tz = np.trapezoid(rho, z, axis=1)
    return r, Tz


_TTAB = None


def thickness(x, y):
    global _TTAB
    if _TTAB is None:
        _TTAB = _thickness_table()
    r, T = _TTAB
    return np.interp(np.sqrt(x * x + y * y), r, T, right=0.0)


def h_eta(eta, eta_w=2.0, sigma_eta=1.8):
    """Longitudinal envelope of Eq. (h_eta)."""
    eta = np.abs(np.asarray(eta, dtype=np.float64))
    d = np.maximum(eta - eta_w, 0.0)
    return np.exp(-d * d / (2 * sigma_eta ** 2))


def n_binary_weight(b):
    """Integral of T_A(x+b/2, y) T_B(x-b/2, y): relative binary-collision count."""
    g = np.linspace(-15, 15, 301)
    X, Y = np.meshgrid(g, g, indexing="ij")
    return float(np.sum(thickness(X + b / 2, Y) * thickness(X - b / 2, Y)) * (g[1] - g[0]) ** 2)


def sample_spots(rng, n_spots, b, eta_max, eta_w=2.0, sigma_eta=1.8):
    """Spot centres: transverse by rejection from T_A(x+b/2,y) T_B(x-b/2,y),
    eta_s from H(|eta|), clipped to the grid."""
    fmax = float(thickness(np.array(0.0), np.array(0.0))) ** 2 * 1.0001
    xs, ys = [], []
    lim = WS_R + 4 * WS_A
    while len(xs) < n_spots:
        m = max(4 * (n_spots - len(xs)), 256)
        x = rng.uniform(-lim, lim, m)
        y = rng.uniform(-lim, lim, m)
        f = thickness(x + b / 2, y) * thickness(x - b / 2, y)
        acc = rng.uniform(0, fmax, m) < f
        xs.extend(x[acc].tolist())
        ys.extend(y[acc].tolist())
    xs = np.array(xs[:n_spots])
    ys = np.array(ys[:n_spots])
    etas = []
    while len(etas) < n_spots:
        m = max(4 * (n_spots - len(etas)), 256)
        e = rng.uniform(0, eta_max, m)
        acc = rng.uniform(0, 1, m) < h_eta(e, eta_w, sigma_eta)
        etas.extend(e[acc].tolist())
    etas = np.array(etas[:n_spots]) * np.where(rng.uniform(size=n_spots) < 0.5, -1.0, 1.0)
    return xs, ys, etas


def deposit_spots(nx, ny, neta, dx, dy, deta, xs, ys, etas, amp, sigma_r=0.6, sigma_eta=0.6,
                  weights=None, chunk=512):
    """Sum of Gaussians sum_s w_s amp exp(-r^2/2 sigma_r^2 - (eta-eta_s)^2/2 sigma_eta^2).
    ``weights`` may be a list of weight vectors: then one field per vector."""
    many = isinstance(weights, (list, tuple))
    wl = list(weights) if many else [weights]
    x = cell_coords(nx, dx)
    y = cell_coords(ny, dy)
    eta = cell_coords(neta, deta)
    xs, ys, etas = (np.asarray(a, dtype=np.float64) for a in (xs, ys, etas))
    wl = [np.ones(len(xs)) if w is None else np.asarray(w, dtype=np.float64) for w in wl]
    outs = [np.zeros((nx * ny, neta)) for _ in wl]
    # each Gaussian is separable: a chunk of spots is one matrix product,
    # (x, y) profiles (cells x spots) times weighted eta profiles (spots x eta)
    for s0 in range(0, len(xs), chunk):
        s1 = min(len(xs), s0 + chunk)
        gx = np.exp(-(x[None, :] - xs[s0:s1, None]) ** 2 / (2 * sigma_r ** 2)) * amp
        gy = np.exp(-(y[None, :] - ys[s0:s1, None]) ** 2 / (2 * sigma_r ** 2))
        ge = np.exp(-(eta[None, :] - etas[s0:s1, None]) ** 2 / (2 * sigma_eta ** 2))
        At = (gx[:, :, None] * gy[:, None, :]).reshape(s1 - s0, nx * ny).T
        for o, w in zip(outs, wl):
            o += At @ (w[s0:s1, None] * ge)
    outs = [o.reshape(nx, ny, neta) for o in outs]
    return outs if many else outs[0]


@dataclass
class HydroCase:
    """A complete seeded event: grid, run parameters, EOS and initial fields."""
    name: str
    nx: int
    ny: int
    neta: int
    dx: float
    dy: float
    deta: float
    tau0: float
    dtau: float
    eta_over_s: float
    eos: dict | None
    eps: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    ueta: np.ndarray
    nsteps: int
    cartesian: bool = False
    periodic: bool = False
    T0: np.ndarray | None = None   # (4, nx, ny, neta) T^{tau mu} initial state (then eps/u are unused)
    pi0: np.ndarray | None = None  # (10, nx, ny, neta) initial pi~ (None: 0)
    taupi_coef: float = 0.0        # b in tau_pi = b eta_v / (eps + P); 0 -> 5
    lambda1_hat: float = 0.0       # lambda_1 = lambda1_hat / eps; 0 -> no lambda_1 term

    @property
    def ncells(self):
        return self.nx * self.ny * self.neta


_EOS_CACHE = {}


def crossover_eos():
    if "x" not in _EOS_CACHE:
        _EOS_CACHE["x"] = crossover_eos_table()
    return _EOS_CACHE["x"]


def hotspot_event(nx=97, ny=97, neta=41, dx=0.2, deta=0.2, b=7.0, n_spots=2048, eps_max=55.0,
                  seed=12345, tau0=0.4, dtau=0.01, eta_over_s=0.08, nsteps=400, eos="crossover",
                  name="viscous hot-spot event"):
    """Gaussian hot spots placed from Woods-Saxon thickness at impact parameter
    b; zero initial velocity and pi; amplitude such that max eps = eps_max."""
    rng = np.random.default_rng(seed)
    eta_half = (neta - 1) / 2.0 * deta
    xs, ys, etas = sample_spots(rng, n_spots, b, eta_half)
    eps = deposit_spots(nx, ny, neta, dx, dx, deta, xs, ys, etas, 1.0)
    eps *= eps_max / eps.max()
    z = np.zeros_like(eps)
    return HydroCase(name, nx, ny, neta, dx, dx, deta, tau0, dtau, eta_over_s,
                     crossover_eos() if eos == "crossover" else None,
                     eps, z.copy(), z.copy(), z.copy(), nsteps)


def minijet_event(nx=261, ny=261, neta=121, dx=0.08, deta=0.1, b=7.0, n_spots=8000, eps_max=55.0,
                  seed=2024, tau0=0.4, dtau=0.005, eta_over_s=0.16, nsteps=400, eos="crossover",
                  pt_mean=1.5, m0=1.0, name="hot-spot event with mini-jet initial flow"):
    """Hot spots (placed as in hotspot_event) that each carry a transverse
    momentum: p_T exponential with mean pt_mean (GeV), azimuth uniform; a spot
    deposits T^{tau mu} proportional to its Gaussian profile times
    (1, p_x / m_T, p_y / m_T, 0), m_T = sqrt(p_T^2 + m0^2).  The common
    amplitude makes max T^{tau tau} = eps_max.  pi = 0; the primitives follow
    from the root solve."""
    rng = np.random.default_rng(seed)
    eta_half = (neta - 1) / 2.0 * deta
    xs, ys, etas = sample_spots(rng, n_spots, b, eta_half)
    pt = rng.exponential(pt_mean, n_spots)
    phi = rng.uniform(0.0, 2.0 * np.pi, n_spots)
    mt = np.sqrt(pt ** 2 + m0 ** 2)
    Ttt, Ttx, Tty = deposit_spots(nx, ny, neta, dx, dx, deta, xs, ys, etas, 1.0,
                                  weights=[None, pt * np.cos(phi) / mt, pt * np.sin(phi) / mt])
    scale = eps_max / Ttt.max()
    T0 = np.stack([Ttt * scale, Ttx * scale, Tty * scale, np.zeros_like(Ttt)])
    z = np.zeros_like(Ttt)
    return HydroCase(name, nx, ny, neta, dx, dx, deta, tau0, dtau, eta_over_s,
                     crossover_eos() if eos == "crossover" else None,
                     z.copy(), z.copy(), z.copy(), z.copy(), nsteps, T0=T0)


def binary_overlap(b, n=201):
    """N_bin(b) up to a constant: the integral of T_A(x + b/2, y) T_B(x - b/2, y)."""
    lim = WS_R + 4 * WS_A + b / 2
    x = np.linspace(-lim, lim, n)
    X, Y = np.meshgrid(x, x, indexing="ij")
    return float((thickness(X + b / 2, Y) * thickness(X - b / 2, Y)).sum() * (x[1] - x[0]) ** 2)


_SPOT_AMP = {}


def spot_amplitude():
    """Per-spot amplitude of the 97x97x41 hot-spot event (seed 12345): the
    factor that makes its max eps 55 GeV/fm^3."""
    if "a" not in _SPOT_AMP:
        rng = np.random.default_rng(12345)
        xs, ys, etas = sample_spots(rng, 2048, 7.0, 20 * 0.2)
        _SPOT_AMP["a"] = 55.0 / deposit_spots(97, 97, 41, 0.2, 0.2, 0.2, xs, ys, etas, 1.0).max()
    return _SPOT_AMP["a"]


def batch_events(n=256, seed0=1000, tau0=0.4, dtau=0.01, eos="crossover", nsteps=200):
    """Event-by-event batch: event k (seed seed0 + k) draws nx = ny odd in
    [65, 129], neta odd in [21, 61], dx uniform in [0.15, 0.3] fm with
    d eta = dx, b uniform in [0, 12] fm and eta/s from {0, 0.08, 0.16}; its
    N_spots = round(2048 N_bin(b) / N_bin(7)) spots carry the per-spot
    amplitude of the 97x97x41 event.  Zero initial velocity and pi."""
    amp = spot_amplitude()
    nb7 = binary_overlap(7.0)
    tab = crossover_eos() if eos == "crossover" else None
    out = []
    for k in range(n):
        rng = np.random.default_rng(seed0 + k)
        nx = int(rng.integers(32, 65)) * 2 + 1
        neta = int(rng.integers(10, 31)) * 2 + 1
        dx = float(rng.uniform(0.15, 0.3))
        b = float(rng.uniform(0.0, 12.0))
        eta_over_s = float(rng.choice([0.0, 0.08, 0.16]))
        n_spots = max(1, int(round(2048 * binary_overlap(b) / nb7)))
        xs, ys, etas = sample_spots(rng, n_spots, b, (neta - 1) / 2.0 * dx)
        eps = deposit_spots(nx, nx, neta, dx, dx, dx, xs, ys, etas, amp)
        z = np.zeros_like(eps)
        out.append(HydroCase(f"batch event {k}", nx, nx, neta, dx, dx, dx, tau0, dtau, eta_over_s, tab,
                             eps, z, z, z, nsteps))
    return out


def gubser_case(dx=0.3, nx=33, neta=9, deta=0.3, dtau=0.02, tau0=1.0, tau1=3.0, q=1.0):
    """Ideal Gubser flow, conformal EOS, eta/s = 0 (the 33x33x9 check)."""
    x = cell_coords(nx, dx)
    eps2, ux2, uy2 = gubser_ideal(tau0, x, x, q)
    rep = lambda a: np.repeat(a[:, :, None], neta, axis=2)
    nsteps = int(round((tau1 - tau0) / dtau))
    return HydroCase("ideal Gubser flow", nx, nx, neta, dx, dx, deta, tau0, dtau, 0.0, None,
                     rep(eps2), rep(ux2), rep(uy2), np.zeros((nx, nx, neta)), nsteps)


def random_smooth_box(rng, nx, ny, neta, eps_mean=5.0, amp=0.3, vamp=0.2, modes=3):
    """Smooth periodic random fields for closed-box runs (Cartesian mode)."""
    def field(a0, a):
        X, Y, Z = np.meshgrid(np.arange(nx) / nx, np.arange(ny) / ny, np.arange(neta) / neta, indexing="ij")
        f = np.full((nx, ny, neta), a0, dtype=np.float64)
        for _ in range(modes):
            kx, ky, kz = rng.integers(0, 2, 3)
            ph = rng.uniform(0, 2 * np.pi)
            f += a * rng.uniform(-1, 1) * np.cos(2 * np.pi * (kx * X + ky * Y + kz * Z) + ph)
        return f
    eps = field(eps_mean, amp * eps_mean)
    ux = field(0.0, vamp)
    uy = field(0.0, vamp)
    ue = field(0.0, vamp)
    return eps, ux, uy, ue


def freezeout_slices(shape=(13, 11, 9), d=(0.3, 0.3, 0.25), tau0=2.0, tau1=2.12, n_blobs=10, seed=0,
                     eps_peak=2.0):
    """Two time slices of a smooth synthetic fluid for the freeze-out surface
    finder: eps is a sum of Gaussian blobs that dilute as tau^(-4/3) while
    their widths grow linearly in tau (a crude expanding fireball, so that
    the surface eps = eps_f has both time-like and space-like parts); u~ and
    pi~ are smooth random fields.  Returns a dict with tau0, tau1, d (dx, dy,
    deta), eps0, eps1 (grids) and f0, f1 ((13,) + grid: u~^x, u~^y, u~^eta,
    pi~ tt tx ty te xx xy xe yy ye ee)."""
    rng = np.random.default_rng(seed)
    nx, ny, ne = shape
    X, Y, Z = np.meshgrid(cell_coords(nx, d[0]), cell_coords(ny, d[1]), cell_coords(ne, d[2]), indexing="ij")
    half = np.array([(n - 1) * dd / 2 for n, dd in zip(shape, d)])
    c = rng.uniform(-0.7, 0.7, (n_blobs, 3)) * half
    sig = rng.uniform(0.25, 0.5, (n_blobs, 3)) * half
    amp = rng.uniform(0.3, 1.0, n_blobs) * eps_peak
    kx = rng.normal(size=(13, 3)) / half
    ph = rng.uniform(0, 2 * np.pi, 13)
    scale = np.concatenate([[0.4] * 3, [0.02] * 10])

    def at(tau):
        g = tau / tau0
        e = np.zeros(shape)
        for b in range(n_blobs):
            r2 = sum(((V - c[b, a]) / (sig[b, a] * g)) ** 2 for a, V in enumerate((X, Y, Z)))
            e += amp[b] * g ** (-4.0 / 3.0) * np.exp(-0.5 * r2)
        f = np.stack([scale[q] * np.sin(kx[q, 0] * X + kx[q, 1] * Y + kx[q, 2] * Z + ph[q] + 0.3 * tau)
                      for q in range(13)])
        return e, f

    e0, f0 = at(tau0)
    e1, f1 = at(tau1)
    return {"tau0": tau0, "tau1": tau1, "d": tuple(d), "eps0": e0, "eps1": e1, "f0": f0, "f1": f1}


def spectra_grid(nY=41, npt=15, nphi=48, Y_max=4.0, pT_max=4.0):
    """The momentum grid of the smooth spectra: nY rapidities uniform in
    [-Y_max, Y_max], npt transverse momenta at the Gauss-Legendre nodes of
    [0, pT_max] GeV and nphi azimuths at the Gauss-Legendre nodes of
    [0, 2 pi] (the paper tabulates 41 x 15 x 48 points with pT and phi at
    Gauss quadrature nodes).  Returns (Y, pT, w_pT, phi, w_phi)."""
    Y = np.linspace(-Y_max, Y_max, nY)
    x, w = np.polynomial.legendre.leggauss(npt)
    pT, wpT = 0.5 * pT_max * (x + 1), 0.5 * pT_max * w
    x, w = np.polynomial.legendre.leggauss(nphi)
    phi, wphi = np.pi * (x + 1), np.pi * w
    return Y, pT, wpT, phi, wphi


def gubser_charge(tau, x, y, q=1.0, n_norm=1.0):
    """Net charge density carried by the ideal Gubser flow of gubser_ideal:
    n = C 4 q^2 / (tau [1 + 2 q^2 (tau^2 + r^2) + q^4 (tau^2 - r^2)^2]), the
    solution of d_mu (tau n u^mu) = 0 for that velocity field (n cosh^2 rho
    tau^3 is constant along the flow).  C is fixed so that n(tau=1 fm, r=0) =
    n_norm (fm^-3)."""
    def raw(t, r2):
        return 4 * q * q / (t * (1 + 2 * q * q * (t * t + r2) + q ** 4 * (t * t - r2) ** 2))
    C = n_norm / raw(1.0, 0.0)
    X, Y = np.meshgrid(x, y, indexing="ij")
    return C * raw(tau, X * X + Y * Y)
