"""Pins for the oracle's equation of state and primitive recovery.

Primitive recovery (Sec. 3: T_ideal = T - pi -> eps, u) is pinned against
  * the conformal closed form eps = sqrt(4E^2 - 3M^2) - E, and
  * a brute-force bisection on the tabulated EOS written here with numpy.interp,
plus the defining identities E = (eps+P) g^2 - P, M = (eps+P) g^2 v.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1802_04449_gb300 import inputs as I

HBARC = 0.1973269804


@pytest.fixture(scope="module")
def eos_table():
    return I.crossover_eos_table()


def make(eos=None, **kw):
    return oracle.Oracle(1, 1, 1, 0.1, 0.1, 0.1, 1.0, 0.01, eos=eos, **kw)


def test_conformal_eos_stefan_boltzmann():
    check_conformal_eos()


def check_conformal_eos(plant=0):
    # Degrees of freedom of a u, d, s quark-gluon gas: 2*8 gluon states and
    # 7/8 * (2 spin * 2 particle/antiparticle * 3 colour * 3 flavour) quark states.
    g = 2 * 8 + 7.0 / 8.0 * (2 * 2 * 3 * 3)
    assert g == 47.5
    o = make(plant=plant)
    for T in (0.1, 0.137, 0.3, 0.6):
        P_sb = g * math.pi ** 2 / 90.0 * T ** 4 / HBARC ** 3   # Stefan-Boltzmann pressure
        eps = 3 * P_sb
        P, Tor, cs2 = o.eos(eps)
        assert P == pytest.approx(P_sb, rel=1e-14)
        assert Tor == pytest.approx(T, rel=1e-14)
        assert cs2 == pytest.approx(1 / 3, rel=1e-15)
    assert o.eos(0.0) == (0.0, 0.0, pytest.approx(1 / 3))


def test_table_eos_interpolation_against_numpy(eos_table):
    check_table_eos(eos_table)


def check_table_eos(eos_table=None, plant=0):
    eos_table = eos_table if eos_table is not None else I.crossover_eos_table()
    o = make(eos_table, plant=plant)
    rng = np.random.default_rng(3)
    lne_nodes = eos_table["lne0"] + eos_table["dlne"] * np.arange(len(eos_table["P"]))
    for lne in rng.uniform(lne_nodes[0], lne_nodes[-1], 400):
        e = math.exp(lne)
        P, T, cs2 = o.eos(e)
        assert P == pytest.approx(np.interp(lne, lne_nodes, eos_table["P"]), rel=1e-11, abs=1e-300)
        assert T == pytest.approx(np.interp(lne, lne_nodes, eos_table["T"]), rel=1e-11)
        assert cs2 == pytest.approx(np.interp(lne, lne_nodes, eos_table["cs2"]), rel=1e-11)
    # exactly at nodes
    for k in (0, 1, 777, 4094):
        P, T, cs2 = o.eos(math.exp(lne_nodes[k]))
        assert P == pytest.approx(eos_table["P"][k], rel=1e-10)
    # conformal continuation above the last node
    etop = math.exp(lne_nodes[-1])
    P, T, cs2 = o.eos(4 * etop)
    assert P == pytest.approx(eos_table["P"][-1] + 3 * etop / 3, rel=1e-12)
    assert cs2 == 1 / 3


def test_crossover_table_is_thermodynamically_consistent(eos_table):
    """Input-side check: monotone P and T, 0 < c_s^2 <= 1/3, T_f = 137 MeV
    crossed once, s = dP/dT = (eps+P)/T."""
    P, T, cs2, e = eos_table["P"], eos_table["T"], eos_table["cs2"], eos_table["eps"]
    assert np.all(np.diff(P) > 0) and np.all(np.diff(T) > 0)
    assert np.all(cs2 > 0) and np.all(cs2 <= 1 / 3 + 1e-15)
    assert np.count_nonzero(np.diff(np.sign(T - 0.137))) == 1
    s_fd = np.gradient(P, T)
    s = (e + P) / T
    mid = slice(100, -100)
    assert np.max(np.abs(s_fd[mid] / s[mid] - 1)) < 2e-3


# reading R13: M above (1 - 1e-3) E is rescaled to (1 - 1e-3) E before the solve
M_CAP = 1.0 - 1e-3


def rand_EM(rng, n):
    E = 10 ** rng.uniform(-5, 3, n)
    frac = np.concatenate([rng.uniform(0, 1, n - 20), 1 - 10 ** rng.uniform(-5, -1.5, 20)])
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    M = frac * E
    return E, M[:, None] * d


def test_prim_solve_conformal_closed_form():
    o = make()
    rng = np.random.default_rng(7)
    E, Mv = rand_EM(rng, 3000)
    for Ei, Mi in zip(E, Mv):
        M = min(np.linalg.norm(Mi), M_CAP * Ei)
        out = o.prim(Ei, *Mi)
        eps_exact = math.sqrt(4 * Ei * Ei - 3 * M * M) - Ei
        if eps_exact < 1e-7:   # below the vacuum cutoff of Sec. 5
            assert out[0] == 0.0 and out[1] == 1.0
            continue
        assert out[0] == pytest.approx(eps_exact, rel=1e-12)
        v_exact = M / (Ei + eps_exact / 3)
        ut = 1 / math.sqrt(1 - v_exact ** 2)
        assert out[1] == pytest.approx(ut, rel=1e-11)
        np.testing.assert_allclose(out[2:5], ut * v_exact * Mi / np.linalg.norm(Mi), rtol=1e-10, atol=1e-14)
        assert 0 <= out[5] <= 100


def _bisect(E, M, P_of):
    lo = np.zeros_like(E)
    hi = M / E
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        f = mid - M / (E + P_of(E - M * mid))
        pos = f > 0
        hi = np.where(pos, mid, hi)
        lo = np.where(pos, lo, mid)
    return 0.5 * (lo + hi)


def test_prim_solve_table_bruteforce_bisection(eos_table):
    o = make(eos_table)
    rng = np.random.default_rng(11)
    E, Mv = rand_EM(rng, 10000)
    M = np.minimum(np.linalg.norm(Mv, axis=1), M_CAP * E)
    lne_nodes = eos_table["lne0"] + eos_table["dlne"] * np.arange(len(eos_table["P"]))
    P_of = lambda e: np.interp(np.log(e), lne_nodes, eos_table["P"])
    v = _bisect(E, M, P_of)
    eps_bf = E - M * v
    got = np.array([o.prim(Ei, *Mi) for Ei, Mi in zip(E, Mv)])
    vac = eps_bf < 1e-7 * (1 - 1e-9)
    assert np.all(got[vac, 0] == 0.0)
    keep = eps_bf > 1e-7 * (1 + 1e-9)
    got, E, Mv, M, v, eps_bf = got[keep], E[keep], Mv[keep], M[keep], v[keep], eps_bf[keep]
    # eps = E - M v loses digits as M/E -> 1: allow ~100 ulp of E there
    assert np.all(np.abs(got[:, 0] - eps_bf) <= 1e-12 * eps_bf + 2e-14 * E)
    g = 1 / np.sqrt(1 - v * v)
    # d gamma / gamma = gamma^2 v dv: the reference v carries ~1e-16 absolute error
    assert np.all(np.abs(got[:, 1] - g) <= 1e-12 * g + 1e-15 * g ** 3)
    # defining identities with numpy's own interpolation
    Pg = P_of(got[:, 0])
    gv = np.linalg.norm(got[:, 2:5], axis=1)          # |u~| = gamma v
    np.testing.assert_allclose((got[:, 0] + Pg) * got[:, 1] ** 2 - Pg, E, rtol=1e-11)
    np.testing.assert_allclose((got[:, 0] + Pg) * got[:, 1] * gv, M, rtol=1e-11)
    # u~ points along M
    np.testing.assert_allclose(got[:, 2:5] / gv[:, None], Mv / np.linalg.norm(Mv, axis=1)[:, None], atol=1e-12)
    assert got[:, 5].max() <= 100


def test_prim_solve_edge_cases(eos_table):
    for eos in (None, eos_table):
        o = make(eos)
        out = o.prim(5.0, 0.0, 0.0, 0.0)          # at rest
        assert out[0] == 5.0 and out[1] == 1.0 and np.all(out[2:5] == 0)
        out = o.prim(5e-8, 1e-8, 0, 0)            # below the vacuum cutoff
        assert out[0] == 0.0 and out[1] == 1.0
        out = o.prim(2.0, 3.0, 0.0, 0.0)          # M > E: rescaled to (1-1e-3) E
        assert np.isfinite(out).all() and out[0] > 0 and out[2] > 0
        o2 = make(eos)
        ref = o2.prim(2.0, 2.0 * M_CAP, 0.0, 0.0)
        np.testing.assert_allclose(out[:5], ref[:5], rtol=1e-13)
        # just below the bound nothing is rescaled; just above, M is moved onto it
        below = o2.prim(2.0, 2.0 * M_CAP * (1 - 1e-9), 0.0, 0.0)
        above = o2.prim(2.0, 2.0 * M_CAP * (1 + 1e-9), 0.0, 0.0)
        np.testing.assert_allclose(above[:5], ref[:5], rtol=1e-13)
        assert below[0] > ref[0] and abs(below[0] / ref[0] - 1) < 1e-5
