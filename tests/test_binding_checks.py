"""The Python binding refuses device arguments whose size or device does not
match the handle before any C call (the C entry points take plain pointers
and trust the sizes they imply).  CPU: the checks themselves, on stand-in
handles; the GPU tests run the same checks on CUDA tensors."""
import types

import pytest
import torch

from paper_1802_04449_gb300 import clv


def test_check_device_arg():
    clv.check_device_arg(6, 0, 6, 0, "eps")
    clv.check_device_arg(7, 1, 6, 1, "buf", at_least=True)
    with pytest.raises(clv.ClvError):
        clv.check_device_arg(5, 0, 6, 0, "eps")            # too short
    with pytest.raises(clv.ClvError):
        clv.check_device_arg(7, 0, 6, 0, "eps")            # exact size expected
    with pytest.raises(clv.ClvError):
        clv.check_device_arg(5, 0, 6, 0, "buf", at_least=True)
    with pytest.raises(clv.ClvError):
        clv.check_device_arg(6, 1, 6, 0, "eps")            # another device
    with pytest.raises(clv.ClvError):
        clv.check_device_arg(6, None, 6, 0, "eps")         # host memory


def _stand_in(n=24):
    return types.SimpleNamespace(torch=torch, _dev_index=0, N=n, _device_arg=None)


def test_device_arg_refuses_size_and_host_memory():
    h = _stand_in()
    with pytest.raises(clv.ClvError, match="values"):
        clv.Hydro._device_arg(h, torch.zeros(23, dtype=torch.float64), 24, "eps")
    with pytest.raises(clv.ClvError, match="device"):
        clv.Hydro._device_arg(h, torch.zeros(24, dtype=torch.float64), 24, "eps")   # a CPU tensor


def test_mlp_forward_refuses_feature_shape():
    h = _stand_in()
    h._device_arg = lambda a, c, w, d=None: clv.Hydro._device_arg(h, a, c, w, d)
    with pytest.raises(clv.ClvError, match="rows, 10"):
        clv.Hydro.mlp_forward(h, torch.zeros((3, 9)))
    with pytest.raises(clv.ClvError, match="device"):
        clv.Hydro.mlp_forward(h, torch.zeros((3, 10)))           # host memory


def test_freezeout_find_refuses_short_or_mistyped_slices():
    g = clv.fo_grid((5, 4, 3), 0.1, 0.1, 0.1, clv.CLV_FP32)
    finder = types.SimpleNamespace(grid=g, torch=torch, device=torch.device("cuda", 0))
    def sl(numel, dtype=torch.float32, dev=0):
        return clv.FoSlice(1.0, None, [None] * 3, extent=(numel, dev, dtype))
    with pytest.raises(clv.ClvError, match="values"):
        clv.FreezeoutFinder.find(finder, sl(59), sl(60), 0.5)                  # 5 x 4 x 3 = 60 needed
    with pytest.raises(clv.ClvError, match="precision"):
        clv.FreezeoutFinder.find(finder, sl(60, torch.float64), sl(60), 0.5)
    with pytest.raises(clv.ClvError, match="device"):
        clv.FreezeoutFinder.find(finder, sl(60), sl(60, dev=1), 0.5)
    g.eta_pitch = 4                                                             # rows of 4: 80 values
    with pytest.raises(clv.ClvError, match="values"):
        clv.FreezeoutFinder.find(finder, sl(60), sl(80), 0.5)


def test_cooper_frye_refuses_records_it_cannot_read():
    cf = types.SimpleNamespace(torch=torch, device=torch.device("cuda", 0), p=types.SimpleNamespace(precision=clv.CLV_FP32))
    with pytest.raises(ValueError):
        clv.CooperFrye.spectra(cf, torch.zeros(22, dtype=torch.float32))       # not (n, 22)
    with pytest.raises(clv.ClvError, match="device"):
        clv.CooperFrye.spectra(cf, torch.zeros((4, 22), dtype=torch.float32))  # host memory
