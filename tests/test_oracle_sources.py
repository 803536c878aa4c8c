"""Pins for the oracle's source terms against generic tensor calculus.

The tests compute the Christoffel symbols of the Milne metric
g = diag(1, -1, -1, -tau^2) (Eq. christoffel) from the metric itself, build
covariant derivatives with them, and evaluate the conservative tilde form of
  nabla_mu T^{mu nu} = 0                                  (-> S_T)
  Israel-Stewart shear relaxation with lambda_i = 0         (-> S_pi)
at random cell states.  The tilde variables are taken from their definitions
in Sec. 2 (T~ = tau^{1+n_mu+n_nu} T, pi~ = tau^{n_mu+n_nu} pi, u~ = tau^{n_mu} u,
d~_eta = d_eta/tau with n_eta = 1, else 0).  Nothing here reuses the oracle's
tilde-form algebra; only its per-cell source functions are called.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1802_04449_gb300 import inputs as I

sp = pytest.importorskip("sympy")

HBARC = 0.1973269804
tau, x, y, eta = sp.symbols("tau x y eta", positive=True)
X = [tau, x, y, eta]
NPOW = [0, 0, 0, 1]
PI_ORDER = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]


def christoffel():
    g = sp.diag(1, -1, -1, -tau ** 2)
    gi = g.inv()
    G = [[[sp.simplify(sum(gi[a, d] * (sp.diff(g[d, c], X[b]) + sp.diff(g[d, b], X[c]) - sp.diff(g[b, c], X[d]))
                           for d in range(4)) / 2) for c in range(4)] for b in range(4)] for a in range(4)]
    return g, gi, G


G_METRIC, G_INV, GAMMA = christoffel()


def test_christoffel_symbols_match_paper():
    # Eq. (christoffel): Gamma^tau_{eta eta} = tau, Gamma^eta_{tau eta} = Gamma^eta_{eta tau} = 1/tau
    nz = {(a, b, c): GAMMA[a][b][c] for a in range(4) for b in range(4) for c in range(4) if GAMMA[a][b][c] != 0}
    assert nz == {(0, 3, 3): tau, (3, 0, 3): 1 / tau, (3, 3, 0): 1 / tau}


def random_velocity_field(rng, P0):
    """u^x, u^y, u^eta (Milne components) linear in the coordinates; u^tau from u.u = 1."""
    comps = []
    for c in range(3):
        a0 = rng.uniform(-0.6, 0.6) / (P0[0] if c == 2 else 1.0)
        expr = a0
        for d in range(4):
            expr += rng.uniform(-0.5, 0.5) * (X[d] - P0[d])
        comps.append(expr)
    ux, uy, ue = comps
    ut = sp.sqrt(1 + ux ** 2 + uy ** 2 + tau ** 2 * ue ** 2)
    return [ut, ux, uy, ue]


def at(expr, P0):
    return float(expr.subs({X[i]: P0[i] for i in range(4)}))


def tilde_u_and_du(u, P0):
    ut = [u[m] * tau ** NPOW[m] for m in range(4)]
    u0 = np.array([at(e, P0) for e in ut])
    du = np.zeros((4, 4))
    for a in range(4):
        for b in range(4):
            d = sp.diff(ut[b], X[a])
            if a == 3:
                d = d / tau
            du[a, b] = at(d, P0)
    return u0, du


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_source_T_from_covariant_conservation(seed):
    rng = np.random.default_rng(seed)
    P0 = [rng.uniform(0.5, 2.0), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(-1, 1)]
    u = random_velocity_field(rng, P0)
    e_val = rng.uniform(0.5, 20.0)
    Pp = e_val / 3.0
    pi0 = rng.normal(size=(4, 4)) * 0.1 * e_val
    pi0 = pi0 + pi0.T
    g, gi = G_METRIC, G_INV
    uval = [at(c, P0) for c in u]
    # T^{mu nu} at P0 with constant eps, P, pi (only the point value matters)
    Tm = np.array([[e_val * uval[m] * uval[n] - Pp * (float(gi[m, n].subs(tau, P0[0])) - uval[m] * uval[n])
                    + pi0[m, n] for n in range(4)] for m in range(4)])
    # expected source: (1+n_nu) tau^{n_nu} T^{tau nu} + tau^{1+n_nu} (-Gamma^mu_{mu l} T^{l nu} - Gamma^nu_{mu l} T^{mu l})
    t0 = P0[0]
    Gv = np.array([[[float(sp.sympify(GAMMA[a][b][c]).subs(tau, t0)) for c in range(4)] for b in range(4)] for a in range(4)])
    S_exp = np.zeros(4)
    for nu in range(4):
        chris = -np.einsum("mml,ln->n", Gv, Tm)[nu] - np.einsum("nml,ml->n", Gv, Tm)[nu]
        S_exp[nu] = (1 + NPOW[nu]) * t0 ** NPOW[nu] * Tm[0, nu] + t0 ** (1 + NPOW[nu]) * chris
    # d_tau(tau^{1+n} T^{tau nu}) + tau^{-n_i} d_i(tau^{1+n_i+n} T^{i nu})
    #   = tau^{1+n} d_mu T^{mu nu} + (1+n) tau^n T^{tau nu}, and d_mu T^{mu nu}
    #   is minus the Christoffel terms, so the tilde source is S_exp.
    S_T_exp = S_exp
    o = oracle.Oracle(1, 1, 1, 0.1, 0.1, 0.1, 1.0, 0.01)
    ut, _ = tilde_u_and_du(u, P0)
    piee_t = t0 ** 2 * pi0[3, 3]
    Tte_t = t0 ** 2 * Tm[0, 3]
    got = o.source_T(t0, ut, e_val, piee_t, Tte_t)
    np.testing.assert_allclose(got, S_T_exp, rtol=1e-11, atol=1e-11 * abs(Tm).max())
    assert got[0] < 0  # the sign the paper prints (+T~^{eta eta}/tau) would make this positive


def projector_tensors(uval, gi_num, g_num):
    Delta_uu = gi_num - np.outer(uval, uval)          # Delta^{mu nu}
    u_low = g_num @ uval
    Delta_ud = np.eye(4) - np.outer(uval, u_low)      # Delta^mu_nu
    return Delta_uu, Delta_ud, u_low


@pytest.mark.parametrize("seed", [11, 12, 13, 14, 15])
def test_source_pi_from_covariant_israel_stewart(seed):
    rng = np.random.default_rng(seed)
    P0 = [rng.uniform(0.6, 2.0), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(-1, 1)]
    t0 = P0[0]
    u = random_velocity_field(rng, P0)
    eta_over_s = 0.2
    e_val = rng.uniform(1.0, 30.0)
    P_val = e_val / 3
    T_GeV = float(I.conformal_T(e_val))
    s_dens = (e_val + P_val) / T_GeV                 # fm^-3
    eta_v = eta_over_s * s_dens * HBARC                # GeV / fm^2
    tau_pi = 5 * eta_v / (e_val + P_val)               # fm (tau_pi = 5 eta_v / (T s))

    g_num = np.array(G_METRIC.subs(tau, t0), dtype=float)
    gi_num = np.array(G_INV.subs(tau, t0), dtype=float)
    Gv = np.array([[[float(sp.sympify(GAMMA[a][b][c]).subs(tau, t0)) for c in range(4)] for b in range(4)] for a in range(4)])
    uval = np.array([at(c, P0) for c in u])
    du_plain = np.array([[at(sp.diff(u[b], X[a]), P0) for b in range(4)] for a in range(4)])  # d_a u^b
    nabla = du_plain + np.einsum("bac,c->ab", Gv, uval)      # nabla_a u^b
    nabla_low = nabla @ g_num                                # nabla_a u_b
    theta = np.trace(nabla)
    Du = uval @ nabla                                        # Du^b
    Du_low = g_num @ Du
    D_uu, D_ud, u_low = projector_tensors(uval, gi_num, g_num)
    sym = nabla_low + nabla_low.T
    sigma = D_uu @ sym @ D_uu.T - (2 / 3) * D_uu * np.einsum("ab,ab->", D_uu, nabla_low)
    # random transverse traceless pi^{mu nu}
    A = rng.normal(size=(4, 4)) * 0.05 * e_val
    A = A + A.T
    pi = D_uu @ (g_num @ A @ g_num) @ D_uu.T
    pi = pi - D_uu * np.einsum("ab,ab->", g_num @ pi @ g_num, D_uu) / 3.0
    assert np.allclose(pi @ u_low, 0, atol=1e-12 * abs(pi).max())
    # Israel-Stewart: Delta Delta D pi = (eta_v sigma - pi)/tau_pi - 4/3 pi theta
    RHS = (eta_v * sigma - pi) / tau_pi - (4 / 3) * pi * theta
    # components of D pi along u fixed by preserving u_mu pi^{mu nu} = 0
    Y = -(Du_low @ pi)                                       # u_mu D pi^{mu nu}
    Dpi = RHS + np.outer(uval, D_ud @ Y) + np.outer(D_ud @ Y, uval) + np.outer(uval, uval) * (u_low @ Y)
    # u^l d_l pi^{mu nu} = D pi - u^l Gamma^mu_{l d} pi^{d nu} - u^l Gamma^nu_{l d} pi^{mu d}
    chris = np.einsum("l,mld,dn->mn", uval, Gv, pi) + np.einsum("l,nld,md->mn", uval, Gv, pi)
    conv = Dpi - chris
    # arbitrary spatial derivatives of pi; the time derivative follows from conv
    B = {a: (lambda M: M + M.T)(rng.normal(size=(4, 4)) * 0.1) for a in (1, 2, 3)}
    Btau = (conv - sum(uval[a] * B[a] for a in (1, 2, 3))) / uval[0]
    B[0] = Btau
    pi_field = [[pi[m, n] + sum(B[a][m, n] * (X[a] - P0[a]) for a in range(4)) for n in range(4)] for m in range(4)]
    # conservative tilde LHS: d_tau(u~^tau pi~) + d_x(u~^x pi~) + d_y(u~^y pi~) + d_eta(u~^eta pi~)/tau
    ut_f = [u[m] * tau ** NPOW[m] for m in range(4)]
    S_exp = []
    for (m, n) in PI_ORDER:
        pit = pi_field[m][n] * tau ** (NPOW[m] + NPOW[n])
        lhs = sp.diff(ut_f[0] * pit, tau) + sp.diff(ut_f[1] * pit, x) + sp.diff(ut_f[2] * pit, y) \
            + sp.diff(ut_f[3] * pit, eta) / tau
        S_exp.append(at(lhs, P0))
    S_exp = np.array(S_exp)
    o = oracle.Oracle(1, 1, 1, 0.1, 0.1, 0.1, 1.0, 0.01, eta_over_s=eta_over_s)
    ut, du = tilde_u_and_du(u, P0)
    pit0 = np.array([pi[m, n] * t0 ** (NPOW[m] + NPOW[n]) for (m, n) in PI_ORDER])
    got = o.source_pi(t0, ut, du, pit0, e_val)
    scale = np.abs(S_exp).max()
    np.testing.assert_allclose(got, S_exp, rtol=1e-9, atol=1e-10 * scale)
