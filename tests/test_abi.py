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
