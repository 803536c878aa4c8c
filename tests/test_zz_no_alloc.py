"""clv_field_stats_noalloc: the statistics reduction for callers that cannot
allocate device memory (a fixed budget owned by another framework's pool, or
a loop that must not allocate between its timing points).  Its result must
match what the handle-based clv_get_stats reports for the same state, on
consecutive calls (the shared scratch keeps the previous call's contents, so
a second call checks that nothing stale leaks through).

This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1802_04449_gb300 import clv
from paper_1802_04449_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [clv.CLV_FP32, clv.CLV_FP64])
def test_noalloc_stats_match_get_stats_on_two_calls(precision):
    import torch
    case = I.hotspot_event(nx=41, ny=37, neta=21, n_spots=200, seed=31)
    g = clv.from_case(case, precision)
    g.set_initial(case.eps, case.ux, case.uy, case.ueta)
    volume = case.dx * case.dy * case.deta
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    results = []
    for _ in range(2):
        g.step(7)
        ref = g.stats()                                  # existing entry point
        f = g.get_device(["eps", "Ttt"])
        clv.field_stats_noalloc(f["eps"].reshape(-1), f["Ttt"].reshape(-1), volume, out)
        torch.cuda.synchronize()
        e_tot, eps_max = out.tolist()
        assert e_tot == pytest.approx(ref["E_tot"], rel=1e-12)
        assert eps_max == ref["eps_max"]
        results.append((e_tot, eps_max))
    assert results[0] != results[1]                      # the state moved between the calls


def test_noalloc_limit_and_arguments():
    import torch
    n_max = 8388608
    a = torch.rand(n_max + 1, dtype=torch.float64, device="cuda")
    b = torch.rand(n_max + 1, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(clv.ClvError) as ei:
        clv.field_stats_noalloc(a, b, 1.0, out)          # one cell beyond the limit
    assert ei.value.status == 1 and "8388608" in str(ei.value)
    clv.field_stats_noalloc(a[:n_max], b[:n_max], 0.5, out)   # exactly at the limit
    torch.cuda.synchronize()
    e_tot, eps_max = out.tolist()
    assert e_tot == pytest.approx(0.5 * b[:n_max].sum().item(), rel=1e-12)
    assert eps_max == a[:n_max].max().item()


def test_noalloc_wrapper_refuses_bad_tensors():
    """The C entry point trusts the sizes it is given, so the binding checks
    dtype, contiguity, lengths and device before it calls it."""
    import torch
    a = torch.rand(1000, dtype=torch.float64, device="cuda")
    b = torch.rand(1000, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    bad = [(a.float(), b, out), (a, b[:999], out), (a, b, out[:1]), (a, b.cpu(), out),
           (a[::2], b[::2].contiguous(), out)]
    for x, y, o in bad:
        with pytest.raises(clv.ClvError) as ei:
            clv.field_stats_noalloc(x, y, 1.0, o)
        assert ei.value.status == 1
    clv.field_stats_noalloc(a, b, 1.0, out)   # the good call still works afterwards
    torch.cuda.synchronize()
    assert out[1].item() == a.max().item()
