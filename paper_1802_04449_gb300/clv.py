"""Thin ctypes binding of libclv (include/clv.h).  Argument marshalling only:
every step of the hydro path runs in the library's CUDA kernels.  PyTorch
provides the device workspace and the stream.

There is no CPU fallback: if libclv.so is missing or cannot be loaded, the
first use raises RuntimeError.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libclv.so")

CLV_FP64, CLV_FP32 = 0, 1
CLV_EOS_CONFORMAL, CLV_EOS_TABLE = 0, 1
STATUS = {0: "CLV_OK", 1: "CLV_EINVAL", 2: "CLV_ENOMEM", 3: "CLV_ECUDA", 4: "CLV_EROOT",
          5: "CLV_ENONFINITE", 6: "CLV_ETIMEOUT"}

FIELDS = ["eps", "ux", "uy", "ueta", "Ttt", "Ttx", "Tty", "Tte",
          "pitt", "pitx", "pity", "pite", "pixx", "pixy", "pixe", "piyy", "piye", "piee",
          "upx", "upy", "upe", "Nt", "n", "Pi"]
FIELD_BIT = {k: i for i, k in enumerate(FIELDS)}


class clv_config(ctypes.Structure):
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
        ("precision", ctypes.c_int), ("cartesian", ctypes.c_int), ("periodic", ctypes.c_int),
        ("eps_cut", ctypes.c_double), ("kernel", ctypes.c_int),
        ("taupi_coef", ctypes.c_double), ("lambda1_hat", ctypes.c_double), ("halo_x", ctypes.c_int),
        ("charge", ctypes.c_int),
        ("zeta_over_s", ctypes.c_double),
    ]


class clv_stats(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_double), ("step", ctypes.c_int64),
        ("eps_max", ctypes.c_double), ("T_max", ctypes.c_double), ("E_tot", ctypes.c_double),
        ("n_rescaled", ctypes.c_int64), ("n_rootfail", ctypes.c_int64), ("n_polished", ctypes.c_int64),
        ("n_fp32_nonconverged", ctypes.c_int64), ("n_newton_iters", ctypes.c_int64),
        ("n_newton_cells", ctypes.c_int64), ("n_polish_iters", ctypes.c_int64),
        ("n_newton_warp_max", ctypes.c_int64), ("n_newton_warps", ctypes.c_int64),
        ("error_word", ctypes.c_uint32), ("_pad", ctypes.c_uint32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "_pad"}


class clv_tile_info(ctypes.Structure):
    _fields_ = [("TJ", ctypes.c_int), ("TK", ctypes.c_int), ("CX", ctypes.c_int), ("threads", ctypes.c_int),
                ("blocks", ctypes.c_int), ("smem_bytes", ctypes.c_int), ("ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class clv_fo_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("neta", ctypes.c_int), ("eta_pitch", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("deta", ctypes.c_double),
                ("precision", ctypes.c_int), ("cartesian", ctypes.c_int)]


class clv_fo_slice(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("eps", ctypes.c_void_p), ("u", ctypes.c_void_p * 3),
                ("pi", ctypes.c_void_p * 10)]


FO_NREC = 22
FO_RECORD = ["dS_tau", "dS_x", "dS_y", "dS_eta", "tau", "x", "y", "eta", "ut", "ux", "uy", "ueta",
             "pitt", "pitx", "pity", "pite", "pixx", "pixy", "pixe", "piyy", "piye", "piee"]


class clv_cf_species(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("g", ctypes.c_double), ("stat", ctypes.c_int), ("mu", ctypes.c_double)]


class clv_cf_params(ctypes.Structure):
    _fields_ = [("Tf", ctypes.c_double), ("ePf", ctypes.c_double), ("viscous", ctypes.c_int),
                ("precision", ctypes.c_int)]


CF_MAX_SPECIES = 32
# name: (mass GeV, degeneracy, statistics: -1 Bose-Einstein, +1 Fermi-Dirac)
SPECIES = {"pi+": (0.13957, 1.0, -1), "K+": (0.493677, 1.0, -1), "p": (0.938272, 2.0, 1)}


class ClvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def check_device_arg(numel, device_index, want_numel, want_index, what, at_least=False):
    """Refuse (CLV_EINVAL) a device array argument that has the wrong number
    of values or lies on another device than the handle's: the C entry
    points take plain pointers and trust the sizes they imply."""
    if (numel < want_numel) if at_least else (numel != want_numel):
        raise ClvError(1, f"{what} has {numel} values, {'at least ' if at_least else ''}{want_numel} expected")
    if device_index != want_index:
        raise ClvError(1, f"{what} is on device {device_index}, the handle on device {want_index}")


_lock = threading.Lock()
_lib = None
EXPORTED = ["clv_workspace_bytes", "clv_create", "clv_create_ws", "clv_set_initial",
            "clv_set_initial_device", "clv_step", "clv_get_stats", "clv_get_fields",
            "clv_get_fields_device", "clv_get_time", "clv_enable_kernel_timing", "clv_get_kernel_times",
            "clv_destroy", "clv_last_error", "clv_version", "clv_field_stats_noalloc",
            "clv_set_guess", "clv_set_mlp", "clv_mlp_samples", "clv_mlp_forward", "clv_mlp_loss_grad",
            "clv_mlp_train", "clv_get_tile", "clv_set_tile", "clv_autotune", "clv_set_initial_T",
            "clv_set_initial_T_device", "clv_state_bytes", "clv_get_state", "clv_set_state",
            "clv_create_batch", "clv_batch_size", "clv_batch_set_initial", "clv_batch_get_fields",
            "clv_batch_event_stats", "clv_set_graphs", "clv_slab_halo_bytes", "clv_slab_pack",
            "clv_slab_unpack", "clv_slab_fill_edge", "clv_slab_predictor", "clv_stage",
            "clv_fo_scratch_bytes", "clv_fo_find", "clv_fo_grid_of", "clv_fo_current", "clv_fo_slice_bytes",
            "clv_fo_snapshot", "clv_cf_scratch_bytes", "clv_cf_spectra", "clv_set_initial_n",
            "clv_set_initial_n_device", "clv_batch_set_schedule", "clv_fma_rate"]
CLV_GUESS_PREVIOUS, CLV_GUESS_COLD, CLV_GUESS_MLP, CLV_GUESS_MLP_ALL = 0, 1, 2, 3
MLP_NPARAM = 5124
MLP_PARTIAL_FLOATS = 256 * (MLP_NPARAM + 1)          # CLV_MLP_PARTIAL_FLOATS
MLP_TRAIN_WORK_FLOATS = 3 * MLP_NPARAM + MLP_PARTIAL_FLOATS   # CLV_MLP_TRAIN_WORK_FLOATS


def load(path: str | None = None):
    """Load libclv.so (built by paper_1802_04449_gb300.build).  Raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libclv.so not found at {p}; run paper_1802_04449_gb300.build.build() "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(p)
        P, V = ctypes.c_void_p, ctypes.c_void_p
        D = ctypes.POINTER(ctypes.c_double)
        cfgp = ctypes.POINTER(clv_config)
        lib.clv_workspace_bytes.argtypes = [cfgp, ctypes.POINTER(ctypes.c_size_t)]
        lib.clv_create.argtypes = [cfgp, V, ctypes.POINTER(P)]
        lib.clv_create_ws.argtypes = [cfgp, V, V, ctypes.c_size_t, ctypes.POINTER(P)]
        lib.clv_set_initial.argtypes = [P, D, D, D, D, D]
        lib.clv_set_initial_device.argtypes = [P, V, V, V, V, V]
        lib.clv_set_initial_T.argtypes = [P, D]
        lib.clv_set_initial_T_device.argtypes = [P, V]
        lib.clv_set_initial_n.argtypes = [P, D]
        lib.clv_set_initial_n_device.argtypes = [P, V]
        lib.clv_step.argtypes = [P, ctypes.c_int, ctypes.POINTER(clv_stats)]
        lib.clv_get_stats.argtypes = [P, ctypes.POINTER(clv_stats)]
        lib.clv_get_fields.argtypes = [P, ctypes.c_uint32, D]
        lib.clv_get_fields_device.argtypes = [P, ctypes.c_uint32, V]
        lib.clv_get_time.argtypes = [P, D, ctypes.POINTER(ctypes.c_int64)]
        lib.clv_enable_kernel_timing.argtypes = [P, ctypes.c_int]
        lib.clv_get_kernel_times.argtypes = [P, D, ctypes.POINTER(ctypes.c_int64)]
        lib.clv_field_stats_noalloc.argtypes = [V, V, ctypes.c_int64, ctypes.c_double, V, V]
        F = ctypes.POINTER(ctypes.c_float)
        lib.clv_set_guess.argtypes = [P, ctypes.c_int]
        lib.clv_set_mlp.argtypes = [P, F]
        lib.clv_mlp_samples.argtypes = [P, V, V, V]
        lib.clv_mlp_forward.argtypes = [P, V, ctypes.c_int64, V]
        lib.clv_mlp_loss_grad.argtypes = [V, V, V, ctypes.c_int64, V, V, V, V]
        lib.clv_mlp_train.argtypes = [V, V, V, V, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                      ctypes.c_uint64, ctypes.c_int, V, V]
        lib.clv_set_graphs.argtypes = [P, ctypes.c_int]
        lib.clv_slab_halo_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        lib.clv_slab_pack.argtypes = [P, ctypes.c_int, ctypes.c_int, V]
        lib.clv_slab_unpack.argtypes = [P, ctypes.c_int, ctypes.c_int, V]
        lib.clv_slab_fill_edge.argtypes = [P, ctypes.c_int, ctypes.c_int]
        lib.clv_slab_predictor.argtypes = [P, ctypes.c_int]
        lib.clv_stage.argtypes = [P, ctypes.c_int, ctypes.POINTER(clv_stats)]
        lib.clv_create_batch.argtypes = [cfgp, ctypes.c_int, V, ctypes.POINTER(P)]
        lib.clv_batch_size.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64)]
        lib.clv_batch_set_initial.argtypes = [P, ctypes.c_int, D, D, D, D, D]
        lib.clv_batch_get_fields.argtypes = [P, ctypes.c_int, ctypes.c_uint32, D]
        lib.clv_batch_event_stats.argtypes = [P, ctypes.c_int, ctypes.POINTER(clv_stats)]
        lib.clv_batch_set_schedule.argtypes = [P, ctypes.c_int, ctypes.c_int]
        lib.clv_state_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        lib.clv_get_state.argtypes = [P, V, ctypes.c_size_t]
        lib.clv_set_state.argtypes = [P, V, ctypes.c_size_t]
        TI = ctypes.POINTER(clv_tile_info)
        lib.clv_get_tile.argtypes = [P, TI]
        lib.clv_set_tile.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.clv_autotune.argtypes = [P, ctypes.c_int, ctypes.c_int, TI]
        FG, FS = ctypes.POINTER(clv_fo_grid), ctypes.POINTER(clv_fo_slice)
        lib.clv_fo_scratch_bytes.argtypes = [FG, ctypes.POINTER(ctypes.c_size_t)]
        lib.clv_fo_find.argtypes = [FG, FS, FS, ctypes.c_double, V, V, ctypes.c_int64, V, V, V]
        lib.clv_fo_grid_of.argtypes = [P, FG]
        lib.clv_fo_current.argtypes = [P, FS]
        lib.clv_fo_slice_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        lib.clv_fo_snapshot.argtypes = [P, V, FS]
        CP = ctypes.POINTER(clv_cf_params)
        lib.clv_cf_scratch_bytes.argtypes = [CP, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
        lib.clv_cf_spectra.argtypes = [CP, ctypes.POINTER(clv_cf_species), ctypes.c_int, V, ctypes.c_int64, V,
                                       V, ctypes.c_int, V, ctypes.c_int, V, ctypes.c_int, V, V, V]
        lib.clv_destroy.argtypes = [P]
        lib.clv_destroy.restype = None
        lib.clv_last_error.argtypes = [P]
        lib.clv_last_error.restype = ctypes.c_char_p
        lib.clv_version.restype = ctypes.c_char_p
        lib.clv_fma_rate.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        for name in EXPORTED:
            if name not in ("clv_destroy", "clv_last_error", "clv_version"):
                getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def fma_rate(precision):
    """FMA rate of the current device in TFLOP/s (clv_fma_rate)."""
    lib = load()
    out = ctypes.c_double()
    _raise(lib, lib.clv_fma_rate(int(precision), ctypes.byref(out)))
    return out.value


def _raise(lib, st):
    if st != 0:
        msg = lib.clv_last_error(None)
        raise ClvError(st, msg.decode() if msg else "")


class FoSlice:
    """A time slice for the freeze-out finder: the clv_fo_slice struct and
    the device memory it points into (kept alive here)."""

    def __init__(self, tau, eps, u, pi=None, keep=(), extent=None):
        self.s = clv_fo_slice()
        self.s.tau = float(tau)
        self.s.eps = eps
        for m in range(3):
            self.s.u[m] = u[m]
        for q in range(10):
            self.s.pi[q] = pi[q] if pi is not None else None
        self.keep = list(keep)
        # (values per array, device index, dtype) of a slice made from tensors; None for a handle's slice
        self.extent = extent

    @classmethod
    def from_tensors(cls, tau, eps, u, pi=None):
        """Slice from CUDA tensors (grid-shaped, one dtype): eps, u = (u~^x,
        u~^y, u~^eta), pi = ten pi~ components (tt..ee) or None."""
        ts = [eps, *u] + (list(pi) if pi is not None else [])
        for t in ts:
            if not (t.is_cuda and t.is_contiguous() and t.dtype == eps.dtype and t.shape == eps.shape):
                raise ValueError("slice arrays must be contiguous CUDA tensors of one dtype and shape")
        if not all(t.device == eps.device for t in ts):
            raise ValueError("slice arrays must be on one device")
        ptr = lambda t: ctypes.c_void_p(t.data_ptr())
        return cls(tau, ptr(eps), [ptr(t) for t in u], [ptr(t) for t in pi] if pi is not None else None, keep=ts,
                   extent=(eps.numel(), eps.device.index, eps.dtype))

    @property
    def tau(self):
        return self.s.tau


def fo_grid(shape, dx, dy, deta, precision=CLV_FP64, cartesian=False, eta_pitch=0):
    g = clv_fo_grid()
    g.nx, g.ny, g.neta = (int(n) for n in shape)
    g.eta_pitch = int(eta_pitch)
    g.dx, g.dy, g.deta = float(dx), float(dy), float(deta)
    g.precision, g.cartesian = int(precision), int(bool(cartesian))
    return g


class FreezeoutFinder:
    """clv_fo_find with device buffers kept for one grid: find() enqueues the
    four launches on ``stream``; result() synchronises and returns
    (records (n, 22) tensor view, hypercube indices (n,), n)."""

    def __init__(self, grid, capacity=None, device=None, stream=None):
        import torch
        self.torch = torch
        self._lib = load()
        self.grid = grid
        self.device = torch.device(device or "cuda")
        self.device = torch.device("cuda", self.device.index if self.device.index is not None
                                   else torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        n = ctypes.c_size_t()
        _raise(self._lib, self._lib.clv_fo_scratch_bytes(ctypes.byref(grid), ctypes.byref(n)))
        ncube = (grid.nx - 1) * (grid.ny - 1) * (grid.neta - 1)
        self.capacity = ncube if capacity is None else int(capacity)
        dt = torch.float64 if grid.precision == CLV_FP64 else torch.float32
        self.rec = torch.empty((max(self.capacity, 1), FO_NREC), dtype=dt, device=self.device)
        self.cube = torch.empty(max(self.capacity, 1), dtype=torch.int64, device=self.device)
        self.count = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.scratch = torch.empty(n.value, dtype=torch.uint8, device=self.device)

    def find(self, s0, s1, eps_f):
        V = ctypes.c_void_p
        g = self.grid
        need = g.nx * g.ny * (g.eta_pitch or g.neta)
        dt = self.torch.float64 if g.precision == CLV_FP64 else self.torch.float32
        for sl in (s0, s1):
            if sl.extent is not None:     # a slice made from tensors: its arrays must cover the grid
                numel, dev, dtype = sl.extent
                if dtype != dt:
                    raise ClvError(1, f"slice arrays are {dtype}, the grid's precision needs {dt}")
                check_device_arg(numel, dev, need, self.device.index, "slice array", at_least=True)
        _raise(self._lib, self._lib.clv_fo_find(ctypes.byref(self.grid), ctypes.byref(s0.s), ctypes.byref(s1.s),
                                                float(eps_f), V(self.rec.data_ptr()), V(self.cube.data_ptr()),
                                                self.capacity, V(self.count.data_ptr()),
                                                V(self.scratch.data_ptr()), V(self.stream.cuda_stream)))

    def result(self):
        self.stream.synchronize()
        n = int(self.count.item())
        m = min(n, self.capacity)
        return self.rec[:m], self.cube[:m], n


class CooperFrye:
    """clv_cf_spectra for a list of species on one (Y, pT, phi) grid.
    ``species``: names of SPECIES or (mass, g, stat[, mu]) tuples.
    spectra(rec, nel=None, d_nel=None) enqueues the launches and returns the
    device tensor (n_species, nY, npt, nphi) of dN/(dY pT dpT dphi) in GeV^-2;
    rec is a device tensor of records (rows of FO_NREC values); with d_nel
    (a device int64 tensor, e.g. a finder's count) the element count stays on
    the device and rec's rows are only an upper bound."""

    def __init__(self, species, Y, pT, phi, Tf, ePf=1.0, viscous=True, precision=CLV_FP32, device=None,
                 stream=None):
        import torch
        self.torch = torch
        self._lib = load()
        self.device = torch.device(device or "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        sp = [SPECIES[k] if isinstance(k, str) else tuple(k) for k in species]
        if not 1 <= len(sp) <= CF_MAX_SPECIES:
            raise ValueError(f"1 to {CF_MAX_SPECIES} species per call")
        self.nsp = len(sp)
        self._sp = (clv_cf_species * self.nsp)()
        for z, t in enumerate(sp):
            self._sp[z].mass, self._sp[z].g, self._sp[z].stat = float(t[0]), float(t[1]), int(t[2])
            self._sp[z].mu = float(t[3]) if len(t) > 3 else 0.0
        self.p = clv_cf_params()
        self.p.Tf, self.p.ePf, self.p.viscous, self.p.precision = float(Tf), float(ePf), int(bool(viscous)), int(precision)
        axes = [torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel()).to(self.device) for a in (Y, pT, phi)]
        self.Y, self.pT, self.phi = axes
        self.shape = (self.nsp, len(self.Y), len(self.pT), len(self.phi))
        self.out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        self.scratch = None
        self._cap = -1

    def spectra(self, rec, nel=None, d_nel=None):
        t = self.torch
        V = ctypes.c_void_p
        want = t.float64 if self.p.precision == CLV_FP64 else t.float32
        if rec.dtype != want or not rec.is_contiguous() or rec.dim() != 2 or rec.shape[1] != FO_NREC:
            raise ValueError("records must be a contiguous (n, 22) tensor of the precision's type")
        dev = self.device.index if self.device.index is not None else t.cuda.current_device()
        check_device_arg(rec.numel(), rec.device.index, rec.numel(), dev, "records")
        cap = rec.shape[0] if nel is None else int(nel)
        if not 0 <= cap <= rec.shape[0]:
            raise ClvError(1, f"nel = {cap} outside the {rec.shape[0]} rows of the records")
        if d_nel is not None:
            if d_nel.dtype != t.int64 or d_nel.numel() < 1:
                raise ClvError(1, "d_nel is a device int64 tensor holding the element count")
            check_device_arg(d_nel.numel(), d_nel.device.index, 1, dev, "d_nel", at_least=True)
        if cap != self._cap:
            n = ctypes.c_size_t()
            _raise(self._lib, self._lib.clv_cf_scratch_bytes(ctypes.byref(self.p), cap, self.nsp, *self.shape[1:],
                                                             ctypes.byref(n)))
            self.scratch = t.empty(n.value, dtype=t.uint8, device=self.device)
            self._cap = cap
        _raise(self._lib, self._lib.clv_cf_spectra(
            ctypes.byref(self.p), self._sp, self.nsp, V(rec.data_ptr()) if cap > 0 else None, cap,
            V(d_nel.data_ptr()) if d_nel is not None else None, V(self.Y.data_ptr()), self.shape[1],
            V(self.pT.data_ptr()), self.shape[2], V(self.phi.data_ptr()), self.shape[3], V(self.out.data_ptr()),
            V(self.scratch.data_ptr()), V(self.stream.cuda_stream)))
        return self.out


def fo_find(grid, s0, s1, eps_f, capacity=None, device=None, stream=None):
    """One call of clv_fo_find with fresh buffers: (records, hypercube indices, count)."""
    f = FreezeoutFinder(grid, capacity, device, stream)
    f.find(s0, s1, eps_f)
    return f.result()


def make_config(nx, ny, neta, dx, dy, deta, tau0, dtau, eta_over_s=0.0, eos=None,
                precision=CLV_FP64, cartesian=False, periodic=False, eps_cut=1e-7, kernel=0,
                taupi_coef=0.0, lambda1_hat=0.0, halo_x=0, charge=False, zeta_over_s=0.0):
    c = clv_config()
    c.charge = int(bool(charge))
    c.zeta_over_s = float(zeta_over_s)
    c.taupi_coef, c.lambda1_hat = float(taupi_coef), float(lambda1_hat)
    c.halo_x = int(halo_x)
    c.nx, c.ny, c.neta = int(nx), int(ny), int(neta)
    c.dx, c.dy, c.deta = float(dx), float(dy), float(deta)
    c.tau0, c.dtau, c.eta_over_s = float(tau0), float(dtau), float(eta_over_s)
    keep = []
    if eos is None:
        c.eos_kind = CLV_EOS_CONFORMAL
    else:
        c.eos_kind = CLV_EOS_TABLE
        arrs = [np.ascontiguousarray(eos[k], dtype=np.float64) for k in ("P", "T", "cs2")]
        keep += arrs
        c.eos_n = len(arrs[0])
        c.eos_lne0, c.eos_dlne = float(eos["lne0"]), float(eos["dlne"])
        c.eos_P, c.eos_T, c.eos_cs2 = (_dp(a) for a in arrs)
    c.precision = int(precision)
    c.cartesian, c.periodic = int(bool(cartesian)), int(bool(periodic))
    c.eps_cut = float(eps_cut)
    c.kernel = int(kernel)
    return c, keep


class Hydro:
    """One event on the GPU through the C ABI.  The device workspace is a
    torch uint8 tensor; work goes to ``stream`` (default: torch's current)."""

    def __init__(self, nx, ny, neta, dx, dy, deta, tau0, dtau, eta_over_s=0.0, eos=None,
                 precision=CLV_FP64, cartesian=False, periodic=False, eps_cut=1e-7,
                 stream=None, device=None, torch_workspace=True, kernel=0, taupi_coef=0.0, lambda1_hat=0.0,
                 halo_x=0, charge=False, zeta_over_s=0.0):
        import torch
        self._lib = load()
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self._dev_index = self.device.index if self.device.index is not None else torch.cuda.current_device()
        self.device = torch.device("cuda", self._dev_index)
        self.cfg, self._keep = make_config(nx, ny, neta, dx, dy, deta, tau0, dtau, eta_over_s, eos,
                                           precision, cartesian, periodic, eps_cut, kernel, taupi_coef,
                                           lambda1_hat, halo_x, charge, zeta_over_s)
        self.shape = (int(nx), int(ny), int(neta))
        self.N = int(nx) * int(ny) * int(neta)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = ctypes.c_size_t()
        self._check(self._lib.clv_workspace_bytes(ctypes.byref(self.cfg), ctypes.byref(nbytes)), None)
        self.ws_bytes = nbytes.value
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            if torch_workspace:
                self._ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
                st = self._lib.clv_create_ws(ctypes.byref(self.cfg), ctypes.c_void_p(self.stream.cuda_stream),
                                             ctypes.c_void_p(self._ws.data_ptr()), self.ws_bytes,
                                             ctypes.byref(h))
            else:
                self._ws = None
                st = self._lib.clv_create(ctypes.byref(self.cfg), ctypes.c_void_p(self.stream.cuda_stream),
                                          ctypes.byref(h))
        self._check(st, None)
        self._h = h
        self._started = False

    def _check(self, st, h):
        if st != 0:
            msg = self._lib.clv_last_error(h)
            raise ClvError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.clv_destroy(self._h)
            self._h = None

    __del__ = close

    def _device_arg(self, a, count, what, dtype=None):
        """A CUDA tensor argument as a contiguous tensor of ``count`` values
        (float64 unless ``dtype``) on the handle's device; CLV_EINVAL otherwise."""
        check_device_arg(a.numel(), a.device.index, count, self._dev_index, what)
        return a.to(dtype or self.torch.float64).contiguous()

    def set_initial(self, eps, ux, uy, ueta, pi=None):
        t = self.torch
        if isinstance(eps, t.Tensor) and eps.is_cuda:
            arrs = [self._device_arg(a, self.N, name) for a, name in ((eps, "eps"), (ux, "ux"), (uy, "uy"),
                                                                       (ueta, "ueta"))]
            pi_t = self._device_arg(pi, 10 * self.N, "pi") if pi is not None else None
            self._dev_keep = arrs + ([pi_t] if pi_t is not None else [])
            st = self._lib.clv_set_initial_device(self._h, *(ctypes.c_void_p(a.data_ptr()) for a in arrs),
                                                  ctypes.c_void_p(pi_t.data_ptr()) if pi_t is not None else None)
        else:
            arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(self.shape)) for a in (eps, ux, uy, ueta)]
            pa = None
            if pi is not None:
                pa = np.ascontiguousarray(np.asarray(pi, dtype=np.float64).reshape((10,) + self.shape))
            st = self._lib.clv_set_initial(self._h, *(_dp(a) for a in arrs), _dp(pa) if pa is not None else None)
        self._check(st, self._h)

    def set_initial_T(self, T):
        """Initial state from T^{tau mu} (4 x grid: T^{tau tau}, T^{tau x},
        T^{tau y}, tau T^{tau eta}; pi = 0): host array or CUDA tensor."""
        t = self.torch
        if isinstance(T, t.Tensor) and T.is_cuda:
            a = self._device_arg(T, 4 * self.N, "T")
            self._dev_keep = [a]
            st = self._lib.clv_set_initial_T_device(self._h, ctypes.c_void_p(a.data_ptr()))
        else:
            a = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape((4,) + self.shape))
            st = self._lib.clv_set_initial_T(self._h, _dp(a))
        self._check(st, self._h)

    def set_initial_n(self, n):
        """Net charge density (handle created with charge=True), after the
        initial state: host array or CUDA tensor of the grid's shape."""
        t = self.torch
        if isinstance(n, t.Tensor) and n.is_cuda:
            a = self._device_arg(n, self.N, "n")
            self._dev_keep = [a]
            st = self._lib.clv_set_initial_n_device(self._h, ctypes.c_void_p(a.data_ptr()))
        else:
            a = np.ascontiguousarray(np.asarray(n, dtype=np.float64).reshape(self.shape))
            st = self._lib.clv_set_initial_n(self._h, _dp(a))
        self._check(st, self._h)

    def set_initial_case(self, case):
        """Initial state of an inputs.HydroCase (T^{tau mu} when it has one)."""
        if getattr(case, "T0", None) is not None:
            self.set_initial_T(case.T0)
        else:
            self.set_initial(case.eps, case.ux, case.uy, case.ueta, getattr(case, "pi0", None))

    def step(self, n=1, stats=False):
        s = clv_stats()
        st = self._lib.clv_step(self._h, int(n), ctypes.byref(s) if stats else None)
        self._check(st, self._h)
        return s.as_dict() if stats else None

    def stats(self):
        s = clv_stats()
        self._check(self._lib.clv_get_stats(self._h, ctypes.byref(s)), self._h)
        return s.as_dict()

    def time(self):
        tau = ctypes.c_double()
        step = ctypes.c_int64()
        self._lib.clv_get_time(self._h, ctypes.byref(tau), ctypes.byref(step))
        return tau.value, step.value

    # ---- x-slab (halo_x = 2): halo planes and stage-level stepping
    def halo_bytes(self):
        n = ctypes.c_size_t()
        self._check(self._lib.clv_slab_halo_bytes(self._h, ctypes.byref(n)), self._h)
        return n.value

    def _halo_buffer(self, buf):
        if not (isinstance(buf, self.torch.Tensor) and buf.is_cuda and buf.dtype == self.torch.uint8
                and buf.is_contiguous()):
            raise ClvError(1, "a halo buffer is a contiguous uint8 CUDA tensor")
        check_device_arg(buf.numel(), buf.device.index, self.halo_bytes(), self._dev_index, "halo buffer",
                         at_least=True)
        return ctypes.c_void_p(buf.data_ptr())

    def slab_pack(self, set_, side, buf):
        self._check(self._lib.clv_slab_pack(self._h, int(set_), int(side), self._halo_buffer(buf)), self._h)

    def slab_unpack(self, set_, side, buf):
        self._check(self._lib.clv_slab_unpack(self._h, int(set_), int(side), self._halo_buffer(buf)), self._h)

    def slab_fill_edge(self, set_, side):
        self._check(self._lib.clv_slab_fill_edge(self._h, int(set_), int(side)), self._h)

    def viscous_pending(self):
        """True for a viscous x-slab right after its initial state: the
        first-step predictor still has to run (clv_slab_predictor)."""
        return bool(self.cfg.halo_x) and self.cfg.eta_over_s > 0 and self.time()[1] == 0 and not self._started

    def slab_predictor(self, stage):
        self._check(self._lib.clv_slab_predictor(self._h, int(stage)), self._h)

    def stage(self, stage, stats=False):
        self._started = True
        s = clv_stats()
        self._check(self._lib.clv_stage(self._h, int(stage), ctypes.byref(s) if stats else None), self._h)
        return s.as_dict() if stats else None

    def set_graphs(self, on=True):
        self._check(self._lib.clv_set_graphs(self._h, int(bool(on))), self._h)

    def get_state(self):
        """Checkpoint: the complete evolution state as bytes."""
        n = ctypes.c_size_t()
        self._check(self._lib.clv_state_bytes(self._h, ctypes.byref(n)), self._h)
        buf = ctypes.create_string_buffer(n.value)
        self._check(self._lib.clv_get_state(self._h, buf, n.value), self._h)
        return buf.raw

    def set_state(self, state):
        buf = ctypes.create_string_buffer(bytes(state), len(state))
        self._check(self._lib.clv_set_state(self._h, buf, len(state)), self._h)

    def tile(self):
        t = clv_tile_info()
        self._check(self._lib.clv_get_tile(self._h, ctypes.byref(t)), self._h)
        return t.as_dict()

    def set_tile(self, TJ, TK, CX=0):
        self._check(self._lib.clv_set_tile(self._h, int(TJ), int(TK), int(CX)), self._h)

    def autotune(self, max_candidates=12, reps=3):
        """Time candidate tile shapes on the current state; keep the fastest."""
        t = clv_tile_info()
        self._check(self._lib.clv_autotune(self._h, int(max_candidates), int(reps), ctypes.byref(t)), self._h)
        return t.as_dict()

    def set_guess(self, mode):
        self._check(self._lib.clv_set_guess(self._h, int(mode)), self._h)

    def set_mlp(self, params):
        a = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        if a.size != MLP_NPARAM:
            raise ValueError(f"expected {MLP_NPARAM} parameters")
        self._check(self._lib.clv_set_mlp(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), self._h)

    def mlp_samples(self, X=None, Y=None):
        """Training samples of the current state's non-vacuum cells, in cell
        order: (X, Y) float32 device views (rows x 10, rows x 4).  X and Y,
        if given, are device buffers of at least N rows to write into."""
        t = self.torch
        if X is None:
            X = t.empty((self.N, 10), dtype=t.float32, device=self.device)
            Y = t.empty((self.N, 4), dtype=t.float32, device=self.device)
        if X.shape[0] < self.N or Y.shape[0] < self.N or not (X.is_contiguous() and Y.is_contiguous()):
            raise ValueError("sample buffers need N contiguous rows")
        if X.dtype != t.float32 or Y.dtype != t.float32 or X.dim() != 2 or X.shape[1] != 10 or Y.dim() != 2 \
                or Y.shape[1] != 4:
            raise ClvError(1, "sample buffers are float32 (rows, 10) and (rows, 4)")
        check_device_arg(X.numel(), X.device.index, X.numel(), self._dev_index, "X")
        check_device_arg(Y.numel(), Y.device.index, Y.numel(), self._dev_index, "Y")
        n = t.zeros(1, dtype=t.int64, device=self.device)
        self._check(self._lib.clv_mlp_samples(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                              ctypes.c_void_p(n.data_ptr())), self._h)
        self.stream.synchronize()
        rows = int(n.item())
        return X[:rows], Y[:rows]

    def mlp_forward(self, X):
        t = self.torch
        if X.dim() != 2 or X.shape[1] != 10:
            raise ClvError(1, f"features are (rows, 10), got {tuple(X.shape)}")
        X = self._device_arg(X, X.numel(), "X", t.float32)
        Y = t.empty((X.shape[0], 4), dtype=t.float32, device=self.device)
        self._check(self._lib.clv_mlp_forward(self._h, ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                              ctypes.c_void_p(Y.data_ptr())), self._h)
        return Y

    # ---- freeze-out surface (clv_fo_*)
    def fo_grid(self):
        g = clv_fo_grid()
        self._check(self._lib.clv_fo_grid_of(self._h, ctypes.byref(g)), self._h)
        return g

    def fo_current(self):
        """A slice viewing the current state (valid until the next step)."""
        sl = FoSlice(0.0, None, [None] * 3)
        self._check(self._lib.clv_fo_current(self._h, ctypes.byref(sl.s)), self._h)
        sl.keep.append(self)
        return sl

    def fo_snapshot(self):
        """A device copy of the current slice (eps, u~, pi~ at the handle's tau)."""
        n = ctypes.c_size_t()
        self._check(self._lib.clv_fo_slice_bytes(self._h, ctypes.byref(n)), self._h)
        buf = self.torch.empty(n.value, dtype=self.torch.uint8, device=self.device)
        sl = FoSlice(0.0, None, [None] * 3, keep=[buf])
        self._check(self._lib.clv_fo_snapshot(self._h, ctypes.c_void_p(buf.data_ptr()), ctypes.byref(sl.s)),
                    self._h)
        return sl

    def freezeout(self, eps_f, since, capacity=None):
        """Surface elements of eps = eps_f between the slice `since` (an
        earlier fo_snapshot) and the current state: (records, hypercube
        indices, count); synchronises."""
        f = getattr(self, "_fo_finder", None)
        if f is None or (capacity is not None and f.capacity != capacity):
            f = self._fo_finder = FreezeoutFinder(self.fo_grid(), capacity, self.device, self.stream)
        f.find(since, self.fo_current(), eps_f)
        return f.result()

    def enable_kernel_timing(self, on=True):
        self._check(self._lib.clv_enable_kernel_timing(self._h, int(bool(on))), self._h)

    KERNEL_SLOTS = ("stage1", "recover1", "stage2", "recover2")

    def kernel_times(self):
        """Accumulated device ms and launch counts per kernel slot since the last
        read: dict slot -> (ms, launches); slots as in KERNEL_SLOTS."""
        ms = (ctypes.c_double * 4)()
        n = (ctypes.c_int64 * 4)()
        self._check(self._lib.clv_get_kernel_times(self._h, ms, n), self._h)
        return {k: (ms[i], n[i]) for i, k in enumerate(self.KERNEL_SLOTS)}

    @staticmethod
    def mask_of(names):
        m = 0
        for n in names:
            m |= 1 << FIELD_BIT[n]
        return m

    def get(self, names=None, out=None):
        """Host copy of the named fields: dict name -> (nx, ny, neta) float64.
        ``out`` may be a preallocated (len(names), N) float64 array (pinned or not)."""
        if names is None:
            names = FIELDS[:21] + (["Nt", "n"] if self.cfg.charge else []) + (["Pi"] if self.cfg.zeta_over_s > 0 else [])
        names = list([names] if isinstance(names, str) else names)
        names = sorted(names, key=lambda k: FIELD_BIT[k])
        buf = out if out is not None else np.empty((len(names), self.N), dtype=np.float64)
        self._check(self._lib.clv_get_fields(self._h, self.mask_of(names), _dp(buf)), self._h)
        return {k: buf[i].reshape(self.shape) for i, k in enumerate(names)}

    def get_device(self, names):
        t = self.torch
        names = sorted(list(names), key=lambda k: FIELD_BIT[k])
        out = t.empty((len(names), self.N), dtype=t.float64, device=self.device)
        self._check(self._lib.clv_get_fields_device(self._h, self.mask_of(names),
                                                    ctypes.c_void_p(out.data_ptr())), self._h)
        return {k: out[i].view(self.shape) for i, k in enumerate(names)}


def field_stats_noalloc(d_eps, d_Ttt, cell_volume, d_out, stream=None):
    """E_tot and max eps of device float64 tensors into the device tensor
    ``d_out`` (2 values) without any allocation; see clv_field_stats_noalloc.
    The three tensors must be contiguous float64 CUDA tensors on one device,
    d_Ttt as long as d_eps and d_out at least 2 values long (CLV_EINVAL
    otherwise: the C entry point trusts the sizes it is given)."""
    import torch
    lib = load()
    ts = (d_eps, d_Ttt, d_out)
    if not all(isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()
               for x in ts):
        raise ClvError(1, "d_eps, d_Ttt and d_out must be contiguous float64 CUDA tensors")
    if not (d_eps.device == d_Ttt.device == d_out.device):
        raise ClvError(1, "d_eps, d_Ttt and d_out must be on one device")
    if d_Ttt.numel() != d_eps.numel() or d_out.numel() < 2:
        raise ClvError(1, "d_Ttt must have as many values as d_eps, and d_out at least 2")
    n = d_eps.numel()
    with torch.cuda.device(d_eps.device):   # the scratch address is looked up on the current device
        st = stream if stream is not None else torch.cuda.current_stream(d_eps.device)
        status = lib.clv_field_stats_noalloc(ctypes.c_void_p(d_eps.data_ptr()), ctypes.c_void_p(d_Ttt.data_ptr()),
                                             int(n), float(cell_volume), ctypes.c_void_p(st.cuda_stream),
                                             ctypes.c_void_p(d_out.data_ptr()))
    if status != 0:
        raise ClvError(status, lib.clv_last_error(None).decode())


class Batch(Hydro):
    """Many events of different grids in one handle (clv_create_batch):
    one persistent stage launch and one root-solve launch per stage."""

    def __init__(self, cases, precision=CLV_FP64, stream=None, device=None):
        import torch
        self._lib = load()
        self.torch = torch
        self.device = torch.device(device or "cuda")
        cfgs = (clv_config * len(cases))()
        self._keep = []
        for i, c in enumerate(cases):
            cfg, keep = make_config(c.nx, c.ny, c.neta, c.dx, c.dy, c.deta, c.tau0, c.dtau, c.eta_over_s, c.eos,
                                    precision, taupi_coef=getattr(c, "taupi_coef", 0.0),
                                    lambda1_hat=getattr(c, "lambda1_hat", 0.0))
            cfgs[i] = cfg
            self._keep.append(keep)
        self.shapes = [(c.nx, c.ny, c.neta) for c in cases]
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self._lib.clv_create_batch(cfgs, len(cases), ctypes.c_void_p(self.stream.cuda_stream),
                                            ctypes.byref(h))
        self._check(st, None)
        self._h = h
        n, cells = ctypes.c_int(), ctypes.c_int64()
        self._lib.clv_batch_size(h, ctypes.byref(n), ctypes.byref(cells))
        self.nevents, self.N = n.value, cells.value
        self.shape = (self.N, 1, 1)

    def set_event(self, e, eps, ux, uy, ueta, pi=None):
        shp = self.shapes[e]
        arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(shp)) for a in (eps, ux, uy, ueta)]
        pa = None if pi is None else np.ascontiguousarray(np.asarray(pi, dtype=np.float64).reshape((10,) + shp))
        self._check(self._lib.clv_batch_set_initial(self._h, int(e), *(_dp(a) for a in arrs),
                                                    _dp(pa) if pa is not None else None), self._h)

    def get_event(self, e, names):
        names = sorted(list(names), key=lambda k: FIELD_BIT[k])
        shp = self.shapes[e]
        buf = np.empty((len(names), int(np.prod(shp))), dtype=np.float64)
        self._check(self._lib.clv_batch_get_fields(self._h, int(e), self.mask_of(names), _dp(buf)), self._h)
        return {k: buf[i].reshape(shp) for i, k in enumerate(names)}

    def event_stats(self, e):
        s = clv_stats()
        self._check(self._lib.clv_batch_event_stats(self._h, int(e), ctypes.byref(s)), self._h)
        return s.as_dict()

    def set_schedule(self, max_threads, chunk):
        """Tiling policy of the batch: thread cap per CTA, planes per x chunk."""
        self._check(self._lib.clv_batch_set_schedule(self._h, int(max_threads), int(chunk)), self._h)


def mlp_loss_grad(params, X, Y, stream=None):
    """FP32 loss and gradient of the guess network over device samples."""
    import torch
    lib = load()
    st = stream if stream is not None else torch.cuda.current_stream(params.device)
    g = torch.empty(MLP_NPARAM, dtype=torch.float32, device=params.device)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    work = torch.empty(MLP_PARTIAL_FLOATS, dtype=torch.float32, device=params.device)
    status = lib.clv_mlp_loss_grad(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                   ctypes.c_void_p(Y.data_ptr()), X.shape[0], ctypes.c_void_p(st.cuda_stream),
                                   ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                                   ctypes.c_void_p(work.data_ptr()))
    if status != 0:
        raise ClvError(status, lib.clv_last_error(None).decode())
    return loss, g


def mlp_train(params, work, X, Y, iters, batch=8192, lr=1e-3, seed=1, step0=0, stream=None):
    """Adam training of the guess network on the GPU (params/work updated in
    place; work: MLP_TRAIN_WORK_FLOATS floats, zero before the first call);
    returns the per-step mini-batch losses (device tensor).  Deterministic:
    the same inputs give the same parameters bit for bit."""
    import torch
    lib = load()
    st = stream if stream is not None else torch.cuda.current_stream(params.device)
    loss = torch.zeros(max(iters, 1), dtype=torch.float32, device=params.device)
    status = lib.clv_mlp_train(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(work.data_ptr()),
                               ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), X.shape[0], int(iters),
                               int(batch), float(lr), int(seed), int(step0), ctypes.c_void_p(st.cuda_stream),
                               ctypes.c_void_p(loss.data_ptr()))
    if status != 0:
        raise ClvError(status, lib.clv_last_error(None).decode())
    return loss[:iters]


def from_case(case, precision=CLV_FP64, **kw):
    """Hydro handle for an inputs.HydroCase (grid, spacings, times, EOS)."""
    kw.setdefault("taupi_coef", getattr(case, "taupi_coef", 0.0))
    kw.setdefault("lambda1_hat", getattr(case, "lambda1_hat", 0.0))
    return Hydro(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                 case.eta_over_s, case.eos, precision, case.cartesian, case.periodic, **kw)
