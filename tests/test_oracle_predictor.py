"""Pins of the oracle's velocity predictor (Sec. 3): the shear stage update
takes the time derivative of u from u* = 2u^n - u^{n-1}, and the first step
takes u* from one pi-free step (reading R8), i.e. u^{-1} = 2u^0 - u^1_ideal.

- The stored u^{-1} after the initial state equals 2u^0 minus the velocity
  of a separate ideal (pi-free) oracle run after one step, bit for bit.
- After any step the stored u^{n-1} is the velocity of the step before, bit
  for bit.
- On a smooth viscous flow (the second-order viscous Gubser flow of Sec. 5)
  the extrapolation 2u^n - u^{n-1} misses u^{n+1} by O(h^2): halving the step
  quarters the miss.
"""
import numpy as np

import oracle
from paper_1802_04449_gb300 import inputs as I


def _gubser(dtau, plant=0, nx=31, dx=0.2):
    case = I.gubser_viscous_case(dx=dx, nx=nx, neta=3, deta=0.2, dtau=dtau, tau1=1.2)
    o = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                      case.eta_over_s, None, taupi_coef=case.taupi_coef, lambda1_hat=case.lambda1_hat,
                      plant=plant)
    o.set_initial(case.eps, case.ux, case.uy, case.ueta, case.pi0)
    return case, o


def check_first_step_predictor(plant=0):
    case, ov = _gubser(0.02, plant, nx=15, dx=0.4)
    oi = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau, 0.0, None,
                       plant=plant)
    oi.set_initial(case.eps, case.ux, case.uy, case.ueta)
    oi.step(1)
    assert np.abs(oi.get("ux") - ov.get("ux")).max() > 1e-6      # the flow moves within one step
    for up, u in (("upx", "ux"), ("upy", "uy"), ("upe", "ueta")):
        assert np.array_equal(ov.get(up), 2.0 * ov.get(u) - oi.get(u)), up


def check_velocity_history(plant=0):
    _, o = _gubser(0.02, plant, nx=15, dx=0.4)
    o.step(3)
    u3 = {k: o.get(k) for k in ("ux", "uy", "ueta")}
    o.step(1)
    for up, u in (("upx", "ux"), ("upy", "uy"), ("upe", "ueta")):
        assert np.array_equal(o.get(up), u3[u]), up


def extrapolation_miss(dtau, plant=0):
    case, o = _gubser(dtau, plant)
    o.step(int(round(0.1 / dtau)))                 # to tau = 1.1 fm
    un, up = o.get("ux"), o.get("upx")
    o.step(1)
    x = I.cell_coords(case.nx, case.dx)
    X, Y = np.meshgrid(x, x, indexing="ij")
    core = np.sqrt(X * X + Y * Y) <= 1.5
    return float(np.abs(2.0 * un - up - o.get("ux"))[:, :, 1][core].max())


def check_second_order_extrapolation(plant=0):
    e1, e2 = extrapolation_miss(0.02, plant), extrapolation_miss(0.01, plant)
    assert 3.5 < e1 / e2 < 4.5, (e1, e2)


def test_first_step_predictor_is_one_pi_free_step():
    check_first_step_predictor()


def test_velocity_history_is_the_previous_step():
    check_velocity_history()


def test_predictor_extrapolates_to_second_order():
    check_second_order_extrapolation()
