"""Symmetry pins of the oracle's full viscous evolution (the hot-spot kind of
event, which has no closed-form solution).

A hot-spot initial state made symmetric under x -> -x, y -> -y, eta_s -> -eta_s
and x <-> y evolves with those symmetries: the KT fluxes, the sources and the
root solve of Sec. 3 treat the two sides of a cell and the two transverse
axes alike.  Mirrors must hold bit for bit (every operation has its mirror
image); the x <-> y exchange to rounding (the axes are summed in a fixed
order).  Fields odd under a mirror change sign: u^a along its own axis, and
T^{tau a} and pi^{mu nu} by the number of indices along it.
"""
import numpy as np

import oracle
from paper_1802_04449_gb300 import inputs as I

PI = {"pitt": "tt", "pitx": "tx", "pity": "ty", "pite": "te", "pixx": "xx", "pixy": "xy", "pixe": "xe",
      "piyy": "yy", "piye": "ye", "piee": "ee"}
AXIS = {"ux": "x", "uy": "y", "ueta": "e", "Ttx": "x", "Tty": "y", "Tte": "e", "Ttt": "", "eps": ""}
SWAP = {"ux": "uy", "uy": "ux", "Ttx": "Tty", "Tty": "Ttx", "pitx": "pity", "pity": "pitx", "pixx": "piyy",
        "piyy": "pixx", "pixe": "piye", "piye": "pixe"}


def _parity(name, axis):
    idx = PI[name] if name in PI else AXIS[name]
    return -1.0 if idx.count(axis) % 2 else 1.0


def evolve(plant=0, steps=30):
    case = I.hotspot_event(nx=21, ny=21, neta=11, n_spots=40, seed=5, eta_over_s=0.08)
    e = case.eps
    e = e + e[::-1]
    e = e + e[:, ::-1]
    e = e + e[:, :, ::-1]
    e = (e + e.transpose(1, 0, 2)) / 16
    z = np.zeros_like(e)
    o = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                      case.eta_over_s, case.eos, plant=plant)
    o.set_initial(e, z, z, z)
    o.step(steps)
    f = o.fields()
    return {k: f[k] for k in list(AXIS) + list(PI)}


def check_symmetries(plant=0):
    f = evolve(plant)
    assert np.abs(f["ux"]).max() > 1e-2 and np.abs(f["pixy"]).max() > 0   # the flow and the shear have developed
    flips = {"x": lambda a: a[::-1], "y": lambda a: a[:, ::-1], "e": lambda a: a[:, :, ::-1]}
    for ax, flip in flips.items():
        for k, a in f.items():
            assert np.array_equal(flip(a), _parity(k, ax) * a), (ax, k)
    for k, a in f.items():
        b = f[SWAP.get(k, k)].transpose(1, 0, 2)
        scale = np.abs(a).max()
        assert np.abs(a - b).max() <= 1e-13 * scale + 1e-300, ("x<->y", k)


def test_mirror_and_exchange_symmetries_of_a_viscous_event():
    check_symmetries()
