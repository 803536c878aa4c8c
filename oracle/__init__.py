"""FP64 CPU oracle for the CLVisc hydro step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``clv_oracle.c`` (plain C,
FP64, ``-ffp-contract=off``), which shares no code with the CUDA library.

The method it follows and every reading of the paper it takes are listed in
the header of ``clv_oracle.c``.

Parity status per function (what pins it, in ``tests/test_oracle_*.py``):
  eos (conformal)       closed form and thermodynamic identity
  eos (table)           numpy.interp on the same nodes
  prim solve            conformal closed form; brute-force bisection
  S_T, S_pi             generic Christoffel-symbol evaluation of the covariant
                        equations (sympy) at random cell states
  Heun + S_T            ideal Bjorken power law, second-order convergence
  Heun + S_pi           viscous Bjorken ODE (scipy DOP853 at 1e-12)
  KT in Milne + Heun    ideal Gubser flow closed form, convergence
  KT (Cartesian)        Riemann rarefaction closed form, convergence
  KT conservation       periodic Cartesian box, sum T^{t mu} constant
  I^{mu nu}, full step  transversality / trace drift shrinking under refinement
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "clv_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "clv_freezeout.c"), os.path.join(_HERE, "clv_cooperfrye.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libclv_oracle.so")
_lock = threading.Lock()
_libs = {}


def build(force: bool = False, plant: int = 0) -> str:
    """Compile the oracle with gcc (OpenMP, strict FP64 evaluation order).

    ``plant`` > 0 builds a separate copy with one deliberate mistake compiled
    in; only the pin meta-test uses it."""
    os.makedirs(_BUILD, exist_ok=True)
    lib = _LIB if plant == 0 else os.path.join(_BUILD, f"libclv_oracle_plant{plant}.so")
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < max(map(os.path.getmtime, _SRCS)):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-fPIC", "-shared", f"-DPLANT={int(plant)}", "-o", tmp, *_SRCS, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, lib)
    return lib


class _Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("neta", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("deta", ctypes.c_double),
        ("tau0", ctypes.c_double), ("dtau", ctypes.c_double),
        ("eta_over_s", ctypes.c_double),
        ("eos_kind", ctypes.c_int), ("eos_n", ctypes.c_int),
        ("eos_lne0", ctypes.c_double), ("eos_dlne", ctypes.c_double),
        ("eos_P", ctypes.POINTER(ctypes.c_double)),
        ("eos_T", ctypes.POINTER(ctypes.c_double)),
        ("eos_cs2", ctypes.POINTER(ctypes.c_double)),
        ("cartesian", ctypes.c_int), ("periodic", ctypes.c_int),
        ("eps_cut", ctypes.c_double), ("nthreads", ctypes.c_int),
        ("taupi_coef", ctypes.c_double), ("lambda1_hat", ctypes.c_double),
        ("zeta_over_s", ctypes.c_double),
    ]


class _FoGrid(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("neta", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("deta", ctypes.c_double),
        ("tau0", ctypes.c_double), ("tau1", ctypes.c_double), ("cartesian", ctypes.c_int),
    ]


class _CfSpecies(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("g", ctypes.c_double), ("stat", ctypes.c_int),
                ("mu", ctypes.c_double), ("Tf", ctypes.c_double), ("ePf", ctypes.c_double),
                ("viscous", ctypes.c_int)]


def _load(plant: int = 0):
    with _lock:
        if plant not in _libs:
            lib = ctypes.CDLL(build(plant=plant))
            P = ctypes.c_void_p
            D = ctypes.POINTER(ctypes.c_double)
            lib.orc_create.restype = P
            lib.orc_create.argtypes = [ctypes.POINTER(_Config)]
            lib.orc_destroy.argtypes = [P]
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_set_threads.restype = ctypes.c_int
            lib.orc_set_initial.argtypes = [P, D, D, D, D, D]
            lib.orc_set_initial_T.argtypes = [P, D]
            lib.orc_set_initial_n.argtypes = [P, D]
            lib.orc_step.argtypes = [P, ctypes.c_int]
            lib.orc_get.argtypes = [P, ctypes.c_int, D]
            lib.orc_stats.argtypes = [P, D]
            lib.orc_eos.argtypes = [P, ctypes.c_double, D]
            lib.orc_prim.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, D]
            lib.orc_prim_bulk.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, D]
            lib.orc_source_pi.argtypes = [P, ctypes.c_double, D, D, D, ctypes.c_double, D]
            lib.orc_source_T.argtypes = [P, ctypes.c_double, D, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, D]
            G = ctypes.POINTER(_FoGrid)
            lib.orc_freezeout.restype = ctypes.c_int64
            lib.orc_freezeout.argtypes = [G, D, D, D, D, ctypes.c_double, D,
                                          ctypes.POINTER(ctypes.c_int64), ctypes.c_int64]
            lib.orc_cooper_frye.argtypes = [ctypes.POINTER(_CfSpecies), D, ctypes.c_int64, D, ctypes.c_int,
                                            D, ctypes.c_int, D, ctypes.c_int, ctypes.c_int, D]
            lib.orc_freezeout_simplex.argtypes = [G, D, D, ctypes.c_double, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, D]
            _libs[plant] = lib
    return _libs[plant]


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


FIELD_INDEX = {"eps": 0, "ux": 1, "uy": 2, "ueta": 3,
               "Ttt": 4, "Ttx": 5, "Tty": 6, "Tte": 7,
               **{f"pi{k}": 8 + i for i, k in enumerate(
                   ["tt", "tx", "ty", "te", "xx", "xy", "xe", "yy", "ye", "ee"])},
               "upx": 18, "upy": 19, "upe": 20, "Nt": 21, "n": 22, "Pi": 23}


class Oracle:
    """One event on the CPU.  ``eos`` is None (conformal) or a dict with keys
    ``lne0, dlne, P, T, cs2`` (nodes uniform in ln eps)."""

    def __init__(self, nx, ny, neta, dx, dy, deta, tau0, dtau, eta_over_s=0.0, eos=None,
                 cartesian=False, periodic=False, eps_cut=1e-7, nthreads=0, plant=0, taupi_coef=5.0,
                 lambda1_hat=0.0, zeta_over_s=0.0):
        self._lib = _load(plant)
        c = _Config()
        c.nx, c.ny, c.neta = int(nx), int(ny), int(neta)
        c.dx, c.dy, c.deta = float(dx), float(dy), float(deta)
        c.tau0, c.dtau = float(tau0), float(dtau)
        c.eta_over_s = float(eta_over_s)
        self._keep = []
        if eos is None:
            c.eos_kind = 0
        else:
            c.eos_kind = 1
            arrs = [np.ascontiguousarray(eos[k], dtype=np.float64) for k in ("P", "T", "cs2")]
            self._keep += arrs
            c.eos_n = len(arrs[0])
            c.eos_lne0, c.eos_dlne = float(eos["lne0"]), float(eos["dlne"])
            c.eos_P, c.eos_T, c.eos_cs2 = (_dp(a) for a in arrs)
        c.cartesian, c.periodic = int(bool(cartesian)), int(bool(periodic))
        c.eps_cut, c.nthreads = float(eps_cut), int(nthreads)
        c.taupi_coef, c.lambda1_hat = float(taupi_coef), float(lambda1_hat)
        c.zeta_over_s = float(zeta_over_s)
        self.shape = (int(nx), int(ny), int(neta))
        self._h = self._lib.orc_create(ctypes.byref(c))
        if not self._h:
            raise ValueError("oracle rejected the configuration")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    def set_initial(self, eps, ux, uy, ueta, pi=None):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(self.shape) for a in (eps, ux, uy, ueta)]
        pi_arr = None
        if pi is not None:
            pi_arr = np.ascontiguousarray(pi, dtype=np.float64).reshape((10,) + self.shape)
        self._lib.orc_set_initial(self._h, *(_dp(a) for a in arrs),
                                  _dp(pi_arr) if pi_arr is not None else None)

    def set_initial_T(self, T):
        """Initial state from T^{tau mu} (4 x grid: T^{tau tau}, T^{tau x},
        T^{tau y}, tau T^{tau eta}) with pi = 0; primitives by the root solve."""
        a = np.ascontiguousarray(T, dtype=np.float64).reshape((4,) + self.shape)
        if self._lib.orc_set_initial_T(self._h, _dp(a)) != 0:
            raise RuntimeError("root solve hit its iteration cap")

    def set_initial_n(self, n):
        """Net charge density at tau0 (after set_initial): N~^tau = tau0 n u~^tau."""
        a = np.ascontiguousarray(n, dtype=np.float64).reshape(self.shape)
        self._lib.orc_set_initial_n(self._h, _dp(a))

    def step(self, n=1):
        return self._lib.orc_step(self._h, int(n))

    def get(self, name):
        out = np.empty(self.shape, dtype=np.float64)
        if self._lib.orc_get(self._h, FIELD_INDEX[name], _dp(out)) != 0:
            raise KeyError(name)
        return out

    def fields(self):
        return {k: self.get(k) for k in FIELD_INDEX}

    def stats(self):
        out = np.zeros(8)
        self._lib.orc_stats(self._h, _dp(out))
        keys = ["tau", "step", "eps_max", "T_max", "E_tot", "n_rescaled", "n_rootfail", "_"]
        return dict(zip(keys, out.tolist()))

    def eos(self, e):
        out = np.zeros(3)
        self._lib.orc_eos(self._h, float(e), _dp(out))
        return tuple(out)

    def prim(self, E, Mx, My, Me):
        out = np.zeros(6)
        self._lib.orc_prim(self._h, float(E), float(Mx), float(My), float(Me), _dp(out))
        return out

    def prim_bulk(self, E, Mx, My, Me, Pi):
        out = np.zeros(6)
        self._lib.orc_prim_bulk(self._h, float(E), float(Mx), float(My), float(Me), float(Pi), _dp(out))
        return out

    def source_pi(self, tau, u, du, pi, e):
        u = np.ascontiguousarray(u, dtype=np.float64)
        du = np.ascontiguousarray(du, dtype=np.float64).reshape(16)
        pi = np.ascontiguousarray(pi, dtype=np.float64)
        out = np.zeros(10)
        self._lib.orc_source_pi(self._h, float(tau), _dp(u), _dp(du), _dp(pi), float(e), _dp(out))
        return out

    def source_T(self, tau, u, e, piee, Tte):
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.zeros(4)
        self._lib.orc_source_T(self._h, float(tau), _dp(u), float(e), float(piee), float(Tte), _dp(out))
        return out


def set_threads(n: int) -> int:
    return _load().orc_set_threads(int(n))


FO_RECORD = ["dS_tau", "dS_x", "dS_y", "dS_eta", "tau", "x", "y", "eta", "ut", "ux", "uy", "ueta",
             *[f"pi{k}" for k in ("tt", "tx", "ty", "te", "xx", "xy", "xe", "yy", "ye", "ee")]]


def _fo_grid(shape, dx, dy, deta, tau0, tau1, cartesian):
    g = _FoGrid()
    g.nx, g.ny, g.neta = (int(n) for n in shape)
    g.dx, g.dy, g.deta = float(dx), float(dy), float(deta)
    g.tau0, g.tau1, g.cartesian = float(tau0), float(tau1), int(bool(cartesian))
    return g


def freezeout(e0, e1, eps_f, dx, dy, deta, tau0, tau1, fields0=None, fields1=None, cartesian=False,
              capacity=None, plant=0):
    """Surface elements of eps = eps_f between the slices e0 (tau0) and e1
    (tau1), grids of shape (nx, ny, neta); fields*: (13, nx, ny, neta) arrays
    of u~^x, u~^y, u~^eta and pi~ (tt..ee), or None for zeros.  Returns
    (records (n, 22) in FO_RECORD order, hypercube indices (n,)), in
    increasing hypercube order (clv_freezeout.c, readings F1-F6)."""
    e0 = np.ascontiguousarray(e0, dtype=np.float64)
    e1 = np.ascontiguousarray(e1, dtype=np.float64).reshape(e0.shape)
    z = np.zeros((13,) + e0.shape)
    f0 = z if fields0 is None else np.ascontiguousarray(fields0, dtype=np.float64).reshape(z.shape)
    f1 = z if fields1 is None else np.ascontiguousarray(fields1, dtype=np.float64).reshape(z.shape)
    g = _fo_grid(e0.shape, dx, dy, deta, tau0, tau1, cartesian)
    lib = _load(plant)
    if capacity is None:
        capacity = int(np.prod([n - 1 for n in e0.shape]))
    rec = np.zeros((max(capacity, 1), 22))
    cube = np.zeros(max(capacity, 1), dtype=np.int64)
    n = lib.orc_freezeout(ctypes.byref(g), _dp(e0), _dp(e1), _dp(f0), _dp(f1), float(eps_f), _dp(rec),
                          cube.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(capacity))
    if n < 0:
        raise ValueError("bad freeze-out grid")
    m = min(n, capacity)
    return rec[:m].copy(), cube[:m].copy(), int(n)


def freezeout_simplex(e0, e1, eps_f, dx, dy, deta, tau0, tau1, i, j, k, s, cartesian=False, plant=0):
    """dSigma_mu of simplex s (lexicographic ordering of the axes) of
    hypercube (i, j, k) alone."""
    e0 = np.ascontiguousarray(e0, dtype=np.float64)
    e1 = np.ascontiguousarray(e1, dtype=np.float64).reshape(e0.shape)
    g = _fo_grid(e0.shape, dx, dy, deta, tau0, tau1, cartesian)
    out = np.zeros(4)
    _load(plant).orc_freezeout_simplex(ctypes.byref(g), _dp(e0), _dp(e1), float(eps_f), int(i), int(j),
                                       int(k), int(s), _dp(out))
    return out


def cooper_frye(rec, Y, pT, phi, mass, g, stat, Tf, ePf=1.0, mu=0.0, viscous=True, plant=0, absolute=False):
    """dN/(dY pT dpT dphi) (GeV^-2) of one species on the (Y, pT, phi) grid
    from element records (n, 22) in FO_RECORD order (clv_cooperfrye.c,
    readings C1-C4); stat +1 Fermi-Dirac, -1 Bose-Einstein, 0 Boltzmann.
    absolute: the sum of the summands' magnitudes instead (the scale of
    the rounding error of a sum in any order).
    Returns an array of shape (len(Y), len(pT), len(phi))."""
    rec = np.ascontiguousarray(rec, dtype=np.float64).reshape(-1, 22)
    Y, pT, phi = (np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (Y, pT, phi))
    sp = _CfSpecies()
    sp.mass, sp.g, sp.stat, sp.mu = float(mass), float(g), int(stat), float(mu)
    sp.Tf, sp.ePf, sp.viscous = float(Tf), float(ePf), int(bool(viscous))
    out = np.zeros((len(Y), len(pT), len(phi)))
    st = _load(plant).orc_cooper_frye(ctypes.byref(sp), _dp(rec), rec.shape[0], _dp(Y), len(Y), _dp(pT),
                                      len(pT), _dp(phi), len(phi), int(bool(absolute)), _dp(out))
    if st != 0:
        raise ValueError("bad Cooper-Frye arguments")
    return out
