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
