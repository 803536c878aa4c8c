"""Freeze-out surface finder on the GPU (clv_fo_find through the C ABI)
against the FP64 oracle (oracle/clv_freezeout.c), element by element.

Which hypercubes the surface crosses is an integer decision: both sides take
it on the same values (FP32 slices are handed to the oracle as their exact
doubles, eps_f is a float), so the element count and the hypercube indices
must agree exactly, in the same (increasing) order.

Tolerances on the records:
  FP64: 1e-10 relative to the scale of each record column (the largest
        |value| of that column over the surface).
  FP32: 2e-5 of the column scale for dSigma (sums of up to 72 tetrahedra in
        single precision), 1e-5 for positions and interpolated fields.
"""
import numpy as np
import pytest

import oracle
from paper_1802_04449_gb300 import clv
from paper_1802_04449_gb300 import inputs as I

pytestmark = pytest.mark.gpu

PI_NAMES = [f"pi{k}" for k in ("tt", "tx", "ty", "te", "xx", "xy", "xe", "yy", "ye", "ee")]


def _slices(torch, s, dtype, with_pi=True):
    out = []
    for t in (0, 1):
        e = torch.tensor(s[f"eps{t}"], dtype=dtype, device="cuda").contiguous()
        f = [torch.tensor(s[f"f{t}"][q], dtype=dtype, device="cuda").contiguous() for q in range(13)]
        out.append(clv.FoSlice.from_tensors(s[f"tau{t}"], e, f[:3], f[3:] if with_pi else None))
    return out


def _as_used(s, np_dtype):
    """The inputs as the GPU sees them (rounded to the working precision)."""
    r = dict(s)
    for k in ("eps0", "eps1", "f0", "f1"):
        r[k] = s[k].astype(np_dtype).astype(np.float64)
    return r


def _compare(got, ref, fp32):
    assert got.shape == ref.shape
    scale = np.maximum(np.abs(ref).max(axis=0), 1e-30)
    err = np.abs(got - ref) / scale
    if fp32:
        tol = np.full(22, 1e-5)
        tol[:4] = 2e-5
    else:
        tol = np.full(22, 1e-10)
    bad = err > tol
    assert not bad.any(), (np.argwhere(bad)[:5], err.max(axis=0))
    return err.max(axis=0)


def _run(s, eps_f, fp32, with_pi=True, cartesian=False, capacity=None):
    import torch
    dtype = torch.float32 if fp32 else torch.float64
    used = _as_used(s, np.float32 if fp32 else np.float64)
    s0, s1 = _slices(torch, used, dtype, with_pi)
    g = clv.fo_grid(s["eps0"].shape, *s["d"], clv.CLV_FP32 if fp32 else clv.CLV_FP64, cartesian)
    rec, cube, n = clv.fo_find(g, s0, s1, eps_f, capacity=capacity)
    ref, rcube, rn = oracle.freezeout(used["eps0"], used["eps1"], eps_f, *s["d"], s["tau0"], s["tau1"],
                                      used["f0"] if with_pi else np.concatenate([used["f0"][:3], 0 * used["f0"][3:]]),
                                      used["f1"] if with_pi else np.concatenate([used["f1"][:3], 0 * used["f1"][3:]]),
                                      cartesian=cartesian, capacity=capacity)
    assert n == rn
    np.testing.assert_array_equal(cube.cpu().numpy(), rcube)
    return rec.double().cpu().numpy(), ref, n


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("shape", [(13, 11, 9), (37, 29, 23), (2, 2, 2), (5, 3, 2)])
def test_synthetic_slices_match_the_oracle(fp32, shape):
    s = I.freezeout_slices(shape=shape, seed=sum(shape))
    ef = float(np.float32(0.5))
    got, ref, n = _run(s, ef, fp32)
    if shape[0] > 5:
        assert n > 50
    if n:
        _compare(got, ref, fp32)


@pytest.mark.parametrize("fp32", [False, True])
def test_cartesian_and_ideal_slices(fp32):
    s = I.freezeout_slices(shape=(17, 15, 11), seed=4, tau0=0.5, tau1=0.62)
    ef = float(np.float32(0.75))
    got, ref, n = _run(s, ef, fp32, with_pi=False, cartesian=True)
    assert n > 100 and np.all(got[:, 12:] == 0)
    _compare(got, ref, fp32)


def test_ties_capacity_and_empty_surfaces():
    s = I.freezeout_slices(shape=(11, 9, 7), seed=9)
    ef = 0.5
    # corners exactly at eps_f count as inside on both sides
    for k in ("eps0", "eps1"):
        e = s[k].copy()
        e.flat[::7] = ef
        s[k] = e
    got, ref, n = _run(s, ef, False)
    _compare(got, ref, False)
    # a capacity below the count keeps the first records and still counts all
    got2, ref2, n2 = _run(s, ef, False, capacity=13)
    assert n2 == n and got2.shape[0] == 13
    np.testing.assert_array_equal(got2, got[:13])
    # no surface: every corner on one side
    lo = min(s["eps0"].min(), s["eps1"].min())
    hi = max(s["eps0"].max(), s["eps1"].max())
    for v in (0.5 * lo, lo, 2.0 * hi):
        got3, _, n3 = _run(s, v, False)
        assert n3 == 0


def _hydro_pair(precision, nsteps=12):
    case = I.hotspot_event(nx=25, ny=23, neta=11, n_spots=60, seed=5)
    h = clv.from_case(case, precision)
    h.set_initial(case.eps, case.ux, case.uy, case.ueta)
    h.step(20)
    names = ["eps", "ux", "uy", "ueta"] + PI_NAMES
    a = h.get(names)
    tau0 = h.time()[0]
    snap = h.fo_snapshot()
    h.step(nsteps)
    b = h.get(names)
    tau1 = h.time()[0]
    return case, h, snap, a, b, tau0, tau1


@pytest.mark.parametrize("precision", [clv.CLV_FP64, clv.CLV_FP32])
def test_surface_of_a_hydro_run_matches_the_oracle(precision):
    """Slices of the viscous hot-spot event taken by the handle itself
    (padded eta pitch, working precision), against the oracle on the
    exported fields."""
    case, h, snap, a, b, tau0, tau1 = _hydro_pair(precision)
    assert abs(snap.tau - tau0) < 1e-12
    ef = 4.0          # inside the event's range at tau ~ 0.6 fm
    rec, cube, n = h.freezeout(ef, snap)
    f = lambda d: np.stack([d[k] for k in ["ux", "uy", "ueta"] + PI_NAMES])
    ref, rcube, rn = oracle.freezeout(a["eps"], b["eps"], ef, case.dx, case.dy, case.deta, tau0, tau1, f(a), f(b))
    assert n == rn and n > 100
    np.testing.assert_array_equal(cube.cpu().numpy(), rcube)
    _compare(rec.double().cpu().numpy(), ref, precision == clv.CLV_FP32)
    # both kinds of elements appear: time-like (dSigma_tau > 0) and space-like
    assert (ref[:, 0] > 0).any() and (np.abs(ref[:, 1:4]).sum(axis=1) > np.abs(ref[:, 0])).any()
    h.close()


def test_full_size_surface_sampled_against_the_oracle():
    """The 97x97x41 hot-spot event in FP32 (the measured configuration):
    the crossed-hypercube count by brute force over the exported slices, and
    200 sampled elements each recomputed by the oracle on its own 2x2x2
    neighbourhood."""
    case = I.hotspot_event()
    h = clv.from_case(case, clv.CLV_FP32)
    h.set_initial(case.eps, case.ux, case.uy, case.ueta)
    h.step(100)
    names = ["eps", "ux", "uy", "ueta"] + PI_NAMES
    a = h.get(names)
    tau0 = h.time()[0]
    snap = h.fo_snapshot()
    h.step(10)
    b = h.get(names)
    tau1 = h.time()[0]
    ef = float(np.float32(0.25))
    rec, cube, n = h.freezeout(ef, snap)
    e0, e1 = a["eps"], b["eps"]
    nx, ny, ne = e0.shape
    corners = [e[p:p + nx - 1, q:q + ny - 1, r:r + ne - 1] for e in (e0, e1)
               for p in (0, 1) for q in (0, 1) for r in (0, 1)]
    mx, mn = np.max(corners, axis=0), np.min(corners, axis=0)
    want = np.flatnonzero(((mx >= ef) & (mn < ef)).ravel())
    assert n == len(want) and n > 10000
    np.testing.assert_array_equal(cube.cpu().numpy(), want)
    rec = rec.double().cpu().numpy()
    rng = np.random.default_rng(0)
    f = lambda d, sl: np.stack([d[k][sl] for k in ["ux", "uy", "ueta"] + PI_NAMES])
    got, ref = [], []
    for idx in rng.choice(n, 200, replace=False):
        c = int(want[idx])
        i, j, k = c // ((ny - 1) * (ne - 1)), (c // (ne - 1)) % (ny - 1), c % (ne - 1)
        sl = (slice(i, i + 2), slice(j, j + 2), slice(k, k + 2))
        r, _, m = oracle.freezeout(e0[sl], e1[sl], ef, case.dx, case.dy, case.deta, tau0, tau1, f(a, sl), f(b, sl))
        assert m == 1
        r = r[0].copy()
        r[5] += (i + 0.5 - 0.5 * (nx - 1)) * case.dx      # sub-grid centred coordinates -> the event's
        r[6] += (j + 0.5 - 0.5 * (ny - 1)) * case.dy
        r[7] += (k + 0.5 - 0.5 * (ne - 1)) * case.deta
        got.append(rec[idx])
        ref.append(r)
    _compare(np.array(got), np.array(ref), True)
    h.close()
