"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/clv.h declares.  No compute calls (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1802_04449_gb300 import build as B
from paper_1802_04449_gb300 import clv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(clv_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path), path


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["clv_create", "clv_set_initial", "clv_step", "clv_get_fields", "clv_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    so, _ = lib
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing
    assert set(clv.EXPORTED) <= set(declared_functions())


def test_binary_is_sm103a(lib):
    _, path = lib
    data = open(path, "rb").read()
    assert b"sm_103a" in data or b"sm_103" in data


def test_host_only_entry_points(lib):
    so = clv.load()
    assert so.clv_version().decode().startswith("clv-gb300")
    cfg, keep = clv.make_config(97, 97, 41, 0.2, 0.2, 0.2, 0.4, 0.01, 0.08, precision=clv.CLV_FP32)
    n = ctypes.c_size_t()
    assert so.clv_workspace_bytes(ctypes.byref(cfg), ctypes.byref(n)) == 0
    N = 97 * 97 * 41
    assert n.value >= 46 * 4 * N       # 46 FP32 fields per cell
    bad, _ = clv.make_config(0, 1, 1, 0.2, 0.2, 0.2, 0.4, 0.01)
    assert so.clv_workspace_bytes(ctypes.byref(bad), ctypes.byref(n)) == 1
    assert "grid dims" in so.clv_last_error(None).decode()


def test_freezeout_host_checks(lib):
    """clv_fo_scratch_bytes and the argument checks of clv_fo_find run on the
    host (no launch happens when an argument is bad)."""
    so = clv.load()
    g = clv.fo_grid((97, 97, 41), 0.2, 0.2, 0.2, clv.CLV_FP32)
    n = ctypes.c_size_t()
    assert so.clv_fo_scratch_bytes(ctypes.byref(g), ctypes.byref(n)) == 0
    ncube = 96 * 96 * 40
    # a flag byte and a list entry per hypercube, a count and an offset per 256-hypercube block
    assert 5 * ncube <= n.value <= 5 * ncube + 16 * (ncube // 256 + 1) + 128
    assert so.clv_fo_scratch_bytes(ctypes.byref(clv.fo_grid((1, 4, 4), 0.2, 0.2, 0.2)), ctypes.byref(n)) == 1
    assert ">= 2" in so.clv_last_error(None).decode()
    g2 = clv.fo_grid((4, 4, 4), 0.2, 0.2, 0.2, clv.CLV_FP64, eta_pitch=3)
    assert so.clv_fo_scratch_bytes(ctypes.byref(g2), ctypes.byref(n)) == 1
    buf = (ctypes.c_double * 64)()
    p = ctypes.c_void_p(ctypes.addressof(buf))
    s0 = clv.FoSlice(1.0, p, [p, p, p])
    s1 = clv.FoSlice(1.1, p, [p, p, p])
    g = clv.fo_grid((4, 4, 4), 0.2, 0.2, 0.2, clv.CLV_FP64)
    V = ctypes.c_void_p

    def find(a, b, rec=p, cap=1, count=p, scratch=p, ef=0.5):
        return so.clv_fo_find(ctypes.byref(g), ctypes.byref(a.s), ctypes.byref(b.s), ef, rec, None, cap, count,
                              scratch, None)
    assert find(s1, s0) == 1 and "tau" in so.clv_last_error(None).decode()
    assert find(s0, s1, rec=None) == 1 and "d_rec" in so.clv_last_error(None).decode()
    assert find(s0, s1, cap=-1) == 1
    assert find(s0, s1, count=None) == 1
    assert find(s0, s1, scratch=V(ctypes.addressof(buf) + 8)) == 1 and "16-byte" in so.clv_last_error(None).decode()
    assert find(s0, s1, ef=float("nan")) == 1
    s_half = clv.FoSlice(1.1, p, [p, p, p], [p] * 5 + [None] * 5)
    assert find(s0, s_half) == 1 and "pi" in so.clv_last_error(None).decode()
    s_noeps = clv.FoSlice(1.1, None, [p, p, p])
    assert find(s0, s_noeps) == 1 and "eps" in so.clv_last_error(None).decode()
    s_neg = clv.FoSlice(-1.0, p, [p, p, p])
    assert find(s_neg, s1) == 1 and "Milne" in so.clv_last_error(None).decode()


def test_cooperfrye_host_checks(lib):
    """clv_cf_scratch_bytes and the argument checks of clv_cf_spectra run on
    the host (no launch happens when an argument is bad)."""
    so = clv.load()
    p = clv.clv_cf_params()
    p.Tf, p.ePf, p.viscous, p.precision = 0.137, 0.4, 1, clv.CLV_FP32
    n = ctypes.c_size_t()
    assert so.clv_cf_scratch_bytes(ctypes.byref(p), 10000, 3, 41, 15, 48, ctypes.byref(n)) == 0
    assert n.value >= 10000 * 24 * 4 + 3 * 41 * 15 * 48 * 8
    assert so.clv_cf_scratch_bytes(ctypes.byref(p), 10000, 33, 41, 15, 48, ctypes.byref(n)) == 1
    assert "nsp" in so.clv_last_error(None).decode()
    bad = clv.clv_cf_params()
    bad.Tf, bad.ePf, bad.viscous, bad.precision = 0.137, 0.0, 1, clv.CLV_FP32
    assert so.clv_cf_scratch_bytes(ctypes.byref(bad), 10, 1, 4, 4, 4, ctypes.byref(n)) == 1
    assert "ePf" in so.clv_last_error(None).decode()
    buf = (ctypes.c_double * 64)()
    q = ctypes.c_void_p(ctypes.addressof(buf))
    sp = (clv.clv_cf_species * 1)()
    sp[0].mass, sp[0].g, sp[0].stat = 0.14, 1.0, -1

    def call(species=sp, rec=q, out=q, scratch=None, nel=4):
        return so.clv_cf_spectra(ctypes.byref(p), species, 1, rec, nel, None, q, 1, q, 1, q, 1, out, scratch, None)
    assert call() == 1 and "d_scratch" in so.clv_last_error(None).decode()
    assert call(rec=None) == 1 and "d_rec" in so.clv_last_error(None).decode()
    assert call(out=None) == 1 and "d_out" in so.clv_last_error(None).decode()
    sp2 = (clv.clv_cf_species * 1)()
    sp2[0].mass, sp2[0].g, sp2[0].stat = 0.14, 1.0, 2
    assert call(species=sp2) == 1 and "stat" in so.clv_last_error(None).decode()


def test_charge_host_checks(lib):
    """charge = 1 adds two fields to the workspace; a batch or an x-slab with
    charge is refused before anything is allocated."""
    so = clv.load()
    n0, n1 = ctypes.c_size_t(), ctypes.c_size_t()
    c0, _ = clv.make_config(33, 31, 21, 0.2, 0.2, 0.2, 0.4, 0.01, 0.08, precision=clv.CLV_FP32)
    c1, _ = clv.make_config(33, 31, 21, 0.2, 0.2, 0.2, 0.4, 0.01, 0.08, precision=clv.CLV_FP32, charge=True)
    assert so.clv_workspace_bytes(ctypes.byref(c0), ctypes.byref(n0)) == 0
    assert so.clv_workspace_bytes(ctypes.byref(c1), ctypes.byref(n1)) == 0
    assert n1.value - n0.value >= 2 * 33 * 31 * 24 * 4
    cfgs = (clv.clv_config * 1)(c1)
    h = ctypes.c_void_p()
    assert so.clv_create_batch(cfgs, 1, None, ctypes.byref(h)) == 1
    assert "batch" in so.clv_last_error(None).decode()
    c2, _ = clv.make_config(33, 31, 21, 0.2, 0.2, 0.2, 0.4, 0.01, 0.08, halo_x=2, charge=True)
    assert so.clv_workspace_bytes(ctypes.byref(c2), ctypes.byref(n0)) == 1
    assert "x-slab" in so.clv_last_error(None).decode()


def test_bulk_host_checks(lib):
    """zeta_over_s > 0 adds two fields to the workspace; it needs eta_over_s > 0,
    a finite non-negative ratio and a single event (no batch, no x-slab)."""
    so = clv.load()
    n0, n1 = ctypes.c_size_t(), ctypes.c_size_t()
    c0, _ = clv.make_config(33, 31, 21, 0.2, 0.2, 0.2, 0.4, 0.01, 0.08, precision=clv.CLV_FP32)
    c1, _ = clv.make_config(33, 31, 21, 0.2, 0.2, 0.2, 0.4, 0.01, 0.08, precision=clv.CLV_FP32, zeta_over_s=0.05)
    assert so.clv_workspace_bytes(ctypes.byref(c0), ctypes.byref(n0)) == 0
    assert so.clv_workspace_bytes(ctypes.byref(c1), ctypes.byref(n1)) == 0
    assert n1.value - n0.value >= 2 * 33 * 31 * 24 * 4
    for kw, word in [({"eta_over_s": 0.0}, "eta_over_s"), ({"zeta_over_s": -0.1}, "zeta_over_s"),
                     ({"zeta_over_s": float("nan")}, "zeta_over_s"), ({"halo_x": 2}, "x-slab")]:
        args = {"eta_over_s": 0.08, "zeta_over_s": 0.05, **kw}
        c, _ = clv.make_config(33, 31, 21, 0.2, 0.2, 0.2, 0.4, 0.01, **args)
        assert so.clv_workspace_bytes(ctypes.byref(c), ctypes.byref(n0)) == 1, kw
        assert word in so.clv_last_error(None).decode(), kw
    cfgs = (clv.clv_config * 1)(c1)
    h = ctypes.c_void_p()
    assert so.clv_create_batch(cfgs, 1, None, ctypes.byref(h)) == 1
    assert "batch" in so.clv_last_error(None).decode()
