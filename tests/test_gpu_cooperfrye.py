"""Smooth Cooper-Frye spectra on the GPU (clv_cf_spectra through the C ABI)
against the FP64 oracle (oracle/clv_cooperfrye.c), point by point on the
same elements.

Tolerance, per grid point: the rounding error of a sum in any order is
bounded by a multiple of the sum of the summands' magnitudes S (the oracle
returns S too), which exceeds |spectrum| where elements with p.dSigma < 0
cancel others.  So |gpu - oracle| <= tol * S + floor:
  FP64: tol 1e-10, floor 1e-12 of the species' largest S.
  FP32: tol 1e-4 (single-precision products and exp2 of arguments up to
        ~100, summed in FP32 per 128-element tile and in FP64 across tiles),
        floor 1e-20 of the largest S: single-precision terms below ~1e-38 are
        subnormal and lose their relative precision.
"""
import numpy as np
import pytest

import oracle
from paper_1802_04449_gb300 import clv
from paper_1802_04449_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TF = 0.137
EPF = 0.45


def _check(got, ref, tol):
    ref, scale = ref
    assert got.shape == ref.shape
    for z in range(ref.shape[0]):
        floor = (1e-12 if tol < 1e-6 else 1e-20) * scale[z].max()
        err = np.abs(got[z] - ref[z]) / (scale[z] + floor)
        assert err.max() <= tol, (z, err.max(), np.unravel_index(err.argmax(), err.shape))


def _surface(shape=(13, 11, 9), seed=3):
    s = I.freezeout_slices(shape=shape, seed=seed)
    rec, _, n = oracle.freezeout(s["eps0"], s["eps1"], 0.5, *s["d"], s["tau0"], s["tau1"], s["f0"], s["f1"])
    assert n > 50
    return rec


def _run(rec, species, grid, precision, viscous=True, via_count=False):
    import torch
    dt = torch.float64 if precision == clv.CLV_FP64 else torch.float32
    r = torch.tensor(rec, dtype=dt, device="cuda").contiguous()
    Y, pT, phi = grid
    cf = clv.CooperFrye(species, Y, pT, phi, TF, EPF, viscous, precision)
    if via_count:
        cap = torch.cat([r, torch.zeros((7, 22), dtype=dt, device="cuda")])   # rows past the count are ignored
        n = torch.tensor([rec.shape[0]], dtype=torch.int64, device="cuda")
        out = cf.spectra(cap, d_nel=n)
    else:
        out = cf.spectra(r)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _oracle(rec, species, grid, viscous=True):
    """(spectra, sums of the summands' magnitudes)"""
    Y, pT, phi = grid
    out, scale = [], []
    for k in species:
        m, g, st = clv.SPECIES[k] if isinstance(k, str) else k
        out.append(oracle.cooper_frye(rec, Y, pT, phi, m, g, st, TF, EPF, viscous=viscous))
        scale.append(oracle.cooper_frye(rec, Y, pT, phi, m, g, st, TF, EPF, viscous=viscous, absolute=True))
    return np.array(out), np.array(scale)


@pytest.mark.parametrize("precision,tol", [(clv.CLV_FP64, 1e-10), (clv.CLV_FP32, 1e-4)])
@pytest.mark.parametrize("viscous", [True, False])
def test_three_species_on_a_ragged_grid(precision, tol, viscous):
    """pi+, K+ and p in one call; 5 x 3 x 7 points (phi not a multiple of the
    4 points a thread owns), elements of a synthetic surface."""
    rec = _surface()
    grid = (np.linspace(-1.5, 2.0, 5), np.array([0.1, 0.9, 2.3]), np.linspace(0.1, 6.0, 7))
    sp = ["pi+", "K+", "p"]
    if precision == clv.CLV_FP32:
        rec = rec.astype(np.float32).astype(np.float64)
    _check(_run(rec, sp, grid, precision, viscous), _oracle(rec, sp, grid, viscous), tol)


@pytest.mark.parametrize("precision,tol", [(clv.CLV_FP64, 1e-10), (clv.CLV_FP32, 1e-4)])
def test_paper_grid_with_many_element_chunks(precision, tol):
    """The paper's 41 x 15 x 48 grid over ~1500 elements (several 128-element
    tiles and chunks), the element count read on the device."""
    rec = _surface(shape=(31, 27, 13), seed=8)
    assert rec.shape[0] > 1000
    if precision == clv.CLV_FP32:
        rec = rec.astype(np.float32).astype(np.float64)
    Y, pT, _, phi, _ = I.spectra_grid()
    got = _run(rec, ["pi+"], (Y, pT, phi), precision, via_count=True)
    _check(got, _oracle(rec, ["pi+"], (Y, pT, phi)), tol)


def test_no_elements_gives_zero():
    import torch
    cf = clv.CooperFrye(["pi+"], [0.0], [0.5], [0.0, 1.0], TF, EPF, True, clv.CLV_FP32)
    out = cf.spectra(torch.zeros((0, 22), dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == 0)
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = cf.spectra(torch.ones((40, 22), dtype=torch.float32, device="cuda"), d_nel=n)
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == 0)
    # a count beyond the records' rows is refused before the call
    with pytest.raises(clv.ClvError):
        cf.spectra(torch.ones((4, 22), dtype=torch.float32, device="cuda"), nel=5)


def test_spectra_of_the_benchmark_surface():
    """The 97x97x41 hot-spot event in FP32: surface at T_f = 137 MeV between
    tau = 2.4 and 2.5 fm found on the GPU, spectra of pi+ on the paper's
    41 x 15 x 48 grid straight from the finder's device records and count;
    60 sampled points recomputed by the oracle from the same records."""
    import torch
    case = I.hotspot_event()
    h = clv.from_case(case, clv.CLV_FP32)
    h.set_initial(case.eps, case.ux, case.uy, case.ueta)
    h.step(200)
    snap = h.fo_snapshot()
    h.step(10)
    eos = case.eos
    lne = eos["lne0"] + eos["dlne"] * np.arange(len(eos["T"]))
    ef = float(np.float32(np.exp(np.interp(TF, eos["T"], lne))))
    finder = clv.FreezeoutFinder(h.fo_grid(), stream=h.stream)
    finder.find(snap, h.fo_current(), ef)
    Y, pT, _, phi, _ = I.spectra_grid()
    cf = clv.CooperFrye(["pi+"], Y, pT, phi, TF, EPF, True, clv.CLV_FP32, stream=h.stream)
    out = cf.spectra(finder.rec, d_nel=finder.count).cpu().numpy()
    rec, _, n = finder.result()
    assert n > 5000
    rec = rec.double().cpu().numpy()
    rng = np.random.default_rng(1)
    for _ in range(60):
        a, b, c = rng.integers(41), rng.integers(15), rng.integers(48)
        args = (rec, Y[a:a + 1], pT[b:b + 1], phi[c:c + 1], *clv.SPECIES["pi+"], TF, EPF)
        ref = oracle.cooper_frye(*args)[0, 0, 0]
        S = oracle.cooper_frye(*args, absolute=True)[0, 0, 0]
        assert abs(out[0, a, b, c] - ref) <= 1e-4 * S + 1e-20 * np.abs(out).max(), (a, b, c, out[0, a, b, c], ref, S)
    h.close()
