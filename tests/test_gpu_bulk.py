"""Bulk pressure on the GPU (clv_config zeta_over_s > 0; reading R20 of the
oracle) against the oracle, field by field, through the C ABI.

Tolerances: FP64 the bar of every other field, 1e-10 of |o| + 1e-3 max|o|;
FP32 1e-4 relative on eps where eps > 1e-3 GeV/fm^3 (the bar of the shear
path), and |Pi_gpu - Pi_oracle| <= 1e-5 max|Pi| (single-precision sources
summed over the steps of the run; measured 9.4e-7).
"""
import numpy as np
import pytest

import oracle
from paper_1802_04449_gb300 import clv
from paper_1802_04449_gb300 import inputs as I
from test_gpu_parity import compare_fp64, fp32_eps_err

pytestmark = pytest.mark.gpu

ALL = (["eps", "ux", "uy", "ueta", "Ttt", "Ttx", "Tty", "Tte"] + [k for k in clv.FIELDS if k.startswith("pi")] +
       ["upx", "upy", "upe", "Pi"])


def _pair(case, nsteps, precision, zeta_over_s, kernel=0, **kw):
    o = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                      case.eta_over_s, case.eos, case.cartesian, case.periodic, zeta_over_s=zeta_over_s)
    o.set_initial(case.eps, case.ux, case.uy, case.ueta)
    o.step(nsteps)
    g = clv.from_case(case, precision, kernel=kernel, zeta_over_s=zeta_over_s, **kw)
    g.set_initial(case.eps, case.ux, case.uy, case.ueta)
    st = g.step(nsteps, stats=True)
    assert st["error_word"] == 0
    return o, g


@pytest.mark.parametrize("shape,kernel", [((21, 19, 11), 0), ((21, 19, 11), 1), ((9, 7, 5), 0)])
def test_hotspot_bulk_fp64(shape, kernel):
    case = I.hotspot_event(nx=shape[0], ny=shape[1], neta=shape[2], n_spots=30, seed=11, eta_over_s=0.08)
    o, g = _pair(case, 20, clv.CLV_FP64, 0.1, kernel)
    assert np.abs(o.get("Pi")).max() > 1e-3 * np.abs(o.get("eps")).max()
    compare_fp64(o, g, True, ALL)
    g.close()


def test_hotspot_bulk_regulator_fp64():
    """zeta/s = 1 over 80 steps: |Pi| reaches the bound P in some cells."""
    case = I.hotspot_event(nx=15, ny=13, neta=9, n_spots=20, seed=5, eta_over_s=0.08)
    o, g = _pair(case, 80, clv.CLV_FP64, 1.0)
    Pi, e = o.get("Pi"), o.get("eps")
    P = np.vectorize(lambda x: o.eos(x)[0])(e)
    assert np.sum((np.abs(Pi) >= 0.98 * P) & (e > 1e-3)) > 20   # the regulator clamped these cells
    compare_fp64(o, g, True, ALL)
    g.close()


def test_hotspot_bulk_fp32():
    case = I.hotspot_event(nx=21, ny=19, neta=11, n_spots=30, seed=11, eta_over_s=0.08)
    o, g = _pair(case, 20, clv.CLV_FP32, 0.1)
    assert fp32_eps_err(o, g) <= 1e-4
    ref, got = o.get("Pi"), g.get(["Pi"])["Pi"]
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print("fp32 Pi error / max|Pi|:", err)
    assert err <= 1e-5, err
    g.close()


def test_hotspot_bulk_fp32_learned_guess():
    """The learned guess seeds the shifted root solve (the network sees no Pi;
    an untrained one only changes the starting point): same bars as above."""
    from paper_1802_04449_gb300 import learned as L
    case = I.hotspot_event(nx=21, ny=19, neta=11, n_spots=30, seed=11, eta_over_s=0.08)
    o, g = _pair(case, 0, clv.CLV_FP32, 0.1)
    g.set_mlp(L.init_params(0))
    g.set_guess(clv.CLV_GUESS_MLP)
    o.step(20)
    st = g.step(20, stats=True)
    assert st["error_word"] == 0 and st["n_rootfail"] == 0
    assert fp32_eps_err(o, g) <= 1e-4
    ref, got = o.get("Pi"), g.get(["Pi"])["Pi"]
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    g.close()


def test_bjorken_bulk_on_the_gpu():
    """Uniform Bjorken flow with shear and bulk: the GPU equals the oracle (and
    both follow the three-ODE solution the oracle is pinned to)."""
    e0, tau0, dtau, n = 30.0, 0.6, 0.01, 100
    o = oracle.Oracle(4, 4, 4, 0.3, 0.3, 0.3, tau0, dtau, eta_over_s=0.08, zeta_over_s=0.12, periodic=True)
    g = clv.Hydro(4, 4, 4, 0.3, 0.3, 0.3, tau0, dtau, eta_over_s=0.08, zeta_over_s=0.12, periodic=True)
    e = np.full((4, 4, 4), e0)
    z = np.zeros_like(e)
    for h in (o, g):
        h.set_initial(e, z, z, z)
        h.step(n)
    got = g.get(["eps", "Pi", "piee"])
    for k in ("eps", "Pi", "piee"):
        ref = o.get(k)
        assert np.all(np.abs(got[k] - ref) <= 1e-12 * np.abs(ref).max()), k
    assert got["Pi"][0, 0, 0] < 0
    g.close()


def test_sound_wave_with_bulk_on_the_gpu():
    """The linearised sound wave of the oracle's pins (FP64): the wave is 1e-4
    of e0 = 10, so FP64 rounding of the background (~1e-15 absolute) is 1e-11
    of its amplitude; the bar is 1e-10 of each first-order field's amplitude,
    and 1e-10 relative on eps."""
    nx, L, e0, amp = 64, 4.0, 10.0, 1e-4
    dx = L / nx
    x = (np.arange(nx) + 0.5) * dx
    sh = (nx, 1, 1)
    eps = (e0 * (1 + amp * np.cos(2 * np.pi * x / L))).reshape(sh)
    z = np.zeros(sh)
    o = oracle.Oracle(nx, 1, 1, dx, 1.0, 1.0, 0.0, 0.2 * dx, eta_over_s=0.16, zeta_over_s=0.1, cartesian=True,
                      periodic=True)
    g = clv.Hydro(nx, 1, 1, dx, 1.0, 1.0, 0.0, 0.2 * dx, eta_over_s=0.16, zeta_over_s=0.1, cartesian=True,
                  periodic=True)
    for h in (o, g):
        h.set_initial(eps, z, z, z)
        h.step(160)
    names = ["ux", "Ttx", "pixx", "piyy", "piee", "Pi"]
    got = g.get(names + ["eps"])
    for k in names:
        ref = o.get(k)
        assert np.abs(got[k] - ref).max() <= 1e-10 * np.abs(ref).max(), k
    assert np.abs(got["eps"] / o.get("eps") - 1).max() <= 1e-10
    g.close()


@pytest.mark.parametrize("prec", [clv.CLV_FP64, clv.CLV_FP32])
def test_periodic_box_conserves_energy_momentum_with_bulk(prec):
    rng = np.random.default_rng(9)
    nx, ny, ne = 16, 12, 8
    eps, ux, uy, ue = I.random_smooth_box(rng, nx, ny, ne)
    g = clv.Hydro(nx, ny, ne, 0.3, 0.3, 0.3, 0.0, 0.02, eta_over_s=0.1, zeta_over_s=0.2, precision=prec,
                  cartesian=True, periodic=True)
    g.set_initial(eps, ux, uy, ue)
    names = ["Ttt", "Ttx", "Tty", "Tte"]
    q0 = g.get(names)
    g.step(40, stats=True)
    q1 = g.get(names + ["Pi"])
    assert np.abs(q1["Pi"]).max() > 1e-3 * eps.max()
    tol = 1e-12 if prec == clv.CLV_FP64 else 2e-5
    for k in names:
        assert abs(q1[k].sum() - q0[k].sum()) <= tol * abs(q0["Ttt"].sum()), k
    g.close()


def test_checkpoint_graphs_and_reset_with_bulk():
    case = I.hotspot_event(nx=17, ny=15, neta=9, n_spots=20, seed=4, eta_over_s=0.08)
    runs = []
    for graphs in (True, False):
        g = clv.from_case(case, clv.CLV_FP64, zeta_over_s=0.15)
        g.set_graphs(graphs)
        g.set_initial(case.eps, case.ux, case.uy, case.ueta)
        g.step(5)
        state = g.get_state()
        g.step(6)
        a = g.get(["Pi", "eps"])
        g.set_state(state)
        g.step(6)
        b = g.get(["Pi", "eps"])
        for k in a:
            np.testing.assert_array_equal(a[k], b[k])   # restart continues bit for bit
        runs.append(a)
        # a new initial state starts from Pi = 0
        g.set_initial(case.eps, case.ux, case.uy, case.ueta)
        assert np.all(g.get(["Pi"])["Pi"] == 0)
        g.close()
    for k in runs[0]:
        np.testing.assert_array_equal(runs[0][k], runs[1][k])   # graphs replay the same launches
    # the bulk field needs zeta_over_s > 0, and a bulk checkpoint fits only a bulk handle
    h = clv.from_case(case, clv.CLV_FP64)
    h.set_initial(case.eps, case.ux, case.uy, case.ueta)
    with pytest.raises(clv.ClvError):
        h.get(["Pi"])
    with pytest.raises(clv.ClvError):
        h.set_state(state)
    h.close()


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 5), (3, 1, 1), (2, 3, 1), (4, 5, 3)])
def test_degenerate_grids_with_bulk_and_charge(shape):
    """Axes of 1 to 5 cells: every neighbour of the bulk and charge stencils
    is clamped (no interior fast path on short axes); FP64 against the oracle."""
    nx, ny, ne = shape
    rng = np.random.default_rng(sum(shape))
    e = 4.0 + rng.uniform(0, 2, shape)
    z = np.zeros(shape)
    n0 = 0.2 + 0.05 * rng.uniform(-1, 1, shape)
    case = I.HydroCase("tiny", nx, ny, ne, 0.3, 0.3, 0.3, 0.6, 0.02, 0.1, None, e, z, z, z, 5)
    o = oracle.Oracle(nx, ny, ne, 0.3, 0.3, 0.3, 0.6, 0.02, 0.1, zeta_over_s=0.2)
    o.set_initial(e, z, z, z)
    o.set_initial_n(n0)
    o.step(6)
    g = clv.from_case(case, clv.CLV_FP64, zeta_over_s=0.2, charge=True)
    g.set_initial(e, z, z, z)
    g.set_initial_n(n0)
    g.step(6)
    compare_fp64(o, g, True, ALL + ["Nt", "n"])
    g.close()
