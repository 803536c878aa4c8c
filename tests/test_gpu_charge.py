"""Net charge transport on the GPU (clv_config charge = 1, clv_set_initial_n)
against the oracle (reading R19), field by field.

Tolerances: FP64 1e-10 of each field's scale; FP32 1e-4 relative on n where
eps > 1e-3 GeV/fm^3 (the bar of the other fields).
"""
import numpy as np
import pytest

import oracle
from paper_1802_04449_gb300 import clv
from paper_1802_04449_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _charge_profile(shape, seed):
    rng = np.random.default_rng(seed)
    nx, ny, ne = shape
    X, Y, Z = np.meshgrid(np.arange(nx) / nx, np.arange(ny) / ny, np.arange(ne) / ne, indexing="ij")
    n = np.full(shape, 0.2)
    for _ in range(3):
        k = rng.integers(1, 3, 3)
        n += 0.05 * rng.uniform(-1, 1) * np.cos(2 * np.pi * (k[0] * X + k[1] * Y + k[2] * Z) + rng.uniform(0, 6.3))
    return n


def _pair(case, nsteps, precision, n0, **kw):
    o = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                      case.eta_over_s, case.eos, case.cartesian, case.periodic)
    o.set_initial(case.eps, case.ux, case.uy, case.ueta)
    o.set_initial_n(n0)
    o.step(nsteps)
    g = clv.from_case(case, precision, charge=True, **kw)
    g.set_initial(case.eps, case.ux, case.uy, case.ueta)
    g.set_initial_n(n0)
    g.step(nsteps, stats=True)
    return o, g


@pytest.mark.parametrize("shape", [(21, 19, 11), (9, 7, 5)])
def test_hotspot_charge_fp64(shape):
    case = I.hotspot_event(nx=shape[0], ny=shape[1], neta=shape[2], n_spots=30, seed=11)
    n0 = _charge_profile(shape, 1)
    o, g = _pair(case, 20, clv.CLV_FP64, n0)
    got = g.get(["Nt", "n", "eps"])
    for k in ("Nt", "n"):
        ref = o.get(k)
        scale = np.abs(ref).max()
        assert np.abs(got[k] - ref).max() <= 1e-10 * scale, (k, np.abs(got[k] - ref).max(), scale)
    g.close()


def test_hotspot_charge_fp32():
    case = I.hotspot_event(nx=21, ny=19, neta=11, n_spots=30, seed=11)
    n0 = _charge_profile((21, 19, 11), 2)
    o, g = _pair(case, 20, clv.CLV_FP32, n0)
    e = o.get("eps")
    m = e > 1e-3
    ref, got = o.get("n"), g.get(["n"])["n"]
    assert m.sum() > 100
    assert np.max(np.abs(got[m] / ref[m] - 1)) <= 1e-4
    g.close()


def test_gubser_charge_on_the_gpu():
    c = I.gubser_case(dx=0.15, nx=65, neta=1, deta=0.3, dtau=0.015, tau1=1.6)
    x = I.cell_coords(c.nx, c.dx)
    n0 = I.gubser_charge(c.tau0, x, x)[:, :, None]
    o, g = _pair(c, c.nsteps, clv.CLV_FP64, n0)
    ref, got = o.get("n"), g.get(["n"])["n"]
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    # and both near the closed form
    na = I.gubser_charge(g.time()[0], x, x)
    X, Y = np.meshgrid(x, x, indexing="ij")
    core = X ** 2 + Y ** 2 <= 2.5 ** 2
    assert np.abs(got[:, :, 0] - na)[core].sum() / np.abs(na[core]).sum() < 0.03
    g.close()


@pytest.mark.parametrize("precision", [clv.CLV_FP64, clv.CLV_FP32])
def test_charge_is_conserved_in_a_periodic_box(precision):
    rng = np.random.default_rng(5)
    nx, ny, ne = 16, 12, 8
    eps, ux, uy, ue = I.random_smooth_box(rng, nx, ny, ne)
    g = clv.Hydro(nx, ny, ne, 0.3, 0.3, 0.3, 0.0, 0.02, precision=precision, cartesian=True, periodic=True,
                  charge=True)
    g.set_initial(eps, ux, uy, ue)
    g.set_initial_n(_charge_profile((nx, ny, ne), 3))
    q0 = g.get(["Nt"])["Nt"].sum()
    g.step(60, stats=True)
    q1 = g.get(["Nt"])["Nt"].sum()
    tol = 1e-12 if precision == clv.CLV_FP64 else 2e-5
    assert abs(q1 - q0) <= tol * abs(q0), (q0, q1)
    g.close()


def test_checkpoint_graphs_and_reset_with_charge():
    case = I.hotspot_event(nx=17, ny=15, neta=9, n_spots=20, seed=4)
    n0 = _charge_profile((17, 15, 9), 7)
    runs = []
    for graphs in (True, False):
        g = clv.from_case(case, clv.CLV_FP64, charge=True)
        g.set_graphs(graphs)
        g.set_initial(case.eps, case.ux, case.uy, case.ueta)
        g.set_initial_n(n0)
        g.step(5)
        state = g.get_state()
        g.step(6)
        a = g.get(["Nt"])["Nt"]
        g.set_state(state)
        g.step(6)
        b = g.get(["Nt"])["Nt"]
        np.testing.assert_array_equal(a, b)       # restart continues bit for bit
        runs.append(a)
        # a new initial state carries no charge until set_initial_n
        g.set_initial(case.eps, case.ux, case.uy, case.ueta)
        g.step(2)
        assert np.all(g.get(["Nt"])["Nt"] == 0)
        g.close()
    np.testing.assert_array_equal(runs[0], runs[1])   # graphs replay the same launches
    # charge fields need charge = 1
    h = clv.from_case(case, clv.CLV_FP64)
    h.set_initial(case.eps, case.ux, case.uy, case.ueta)
    with pytest.raises(clv.ClvError):
        h.get(["Nt"])
    with pytest.raises(clv.ClvError):
        h.set_initial_n(n0)
    h.close()
