"""Pins of the oracle's initial state from T^{tau mu} (pi = 0): the
primitives it recovers reproduce the input through the perfect-fluid closed
form T^{tau mu} = (eps + P) u^tau u^mu - P g^{tau mu}, and with the
conformal EOS eps equals sqrt(4 E^2 - 3 M^2) - E."""
import numpy as np
import pytest

import oracle
from paper_1802_04449_gb300 import inputs as I


def _oracle(case, eos, plant=0):
    return oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                         case.eta_over_s, eos, nthreads=2, plant=plant)


def _T_of(o, eps, u1, u2, u3):
    """T^{tau mu} (orthonormal eta component) of a perfect fluid, with P from
    the oracle's EOS (pinned on its own elsewhere)."""
    P = np.vectorize(lambda e: o.eos(e)[0])(eps)
    ut = np.sqrt(1 + u1 ** 2 + u2 ** 2 + u3 ** 2)
    w = eps + P
    return np.stack([w * ut * ut - P, w * ut * u1, w * ut * u2, w * ut * u3])


@pytest.mark.parametrize("eos", ["crossover", None])
def test_primitives_reproduce_the_input_T(eos):
    check_reproduce_T(eos)


def check_reproduce_T(eos="crossover", plant=0):
    case = I.hotspot_event(nx=13, ny=11, neta=7, n_spots=25, seed=4, eos=eos)
    rng = np.random.default_rng(8)
    u = [0.6 * rng.uniform(-1, 1, case.eps.shape) for _ in range(3)]
    o = _oracle(case, case.eos, plant)
    T = _T_of(o, case.eps, *u)
    o.set_initial_T(T)
    live = case.eps >= 1e-7
    got = {k: o.get(k) for k in ("eps", "ux", "uy", "ueta")}
    np.testing.assert_allclose(got["eps"][live], case.eps[live], rtol=1e-11)
    for k, ref in zip(("ux", "uy", "ueta"), u):
        np.testing.assert_allclose(got[k][live], ref[live], rtol=1e-10, atol=1e-12)
    assert np.all(got["eps"][~live] == 0)
    # the stored T~^{tau mu} = tau0 x input (tilde scaling of Sec. 2) on live cells
    for m, k in enumerate(("Ttt", "Ttx", "Tty", "Tte")):
        np.testing.assert_allclose(o.get(k)[live], case.tau0 * T[m][live], rtol=1e-10,
                                   atol=1e-12 * np.abs(T[0]).max())


def test_conformal_closed_form_on_minijet_flow():
    case = I.minijet_event(nx=15, ny=13, neta=5, n_spots=30, seed=6, eos=None)
    o = _oracle(case, None)
    o.set_initial_T(case.T0)
    E = case.T0[0]
    M = np.sqrt(case.T0[1] ** 2 + case.T0[2] ** 2 + case.T0[3] ** 2)
    ref = np.sqrt(4 * E ** 2 - 3 * M ** 2) - E
    live = E >= 1e-7
    np.testing.assert_allclose(o.get("eps")[live], ref[live], rtol=1e-12)
    # velocity along M with |v| = M / (E + P), P = eps / 3
    v = M / (E + ref / 3)
    g = 1 / np.sqrt(1 - v ** 2)
    sel = live & (M > 0)
    np.testing.assert_allclose(o.get("ux")[sel], (g * v * case.T0[1] / np.where(M > 0, M, 1))[sel],
                               rtol=1e-10, atol=1e-13)
