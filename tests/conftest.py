import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libclv")
    config.addinivalue_line("markers", "slow: longer CPU-only oracle runs")


def assert_regulator_inactive(f, P, Pi=None):
    """The viscous regulator (oracle reading R18) leaves a state untouched when
    every cell has eps >= 2e-3 GeV/fm^3 (ramp factor 1) and
    |pi~_{mu nu} pi~^{mu nu}| <= eps^2 + 3 P^2 (and |Pi| <= P).  Analytic pins
    call this on the states they compare, so that the regulator, which the
    paper does not have, plays no part in them."""
    import numpy as np
    e = f["eps"]
    assert e.min() >= 2e-3, e.min()
    pp = (f["pitt"] ** 2 - 2 * (f["pitx"] ** 2 + f["pity"] ** 2 + f["pite"] ** 2) + f["pixx"] ** 2
          + f["piyy"] ** 2 + f["piee"] ** 2 + 2 * (f["pixy"] ** 2 + f["pixe"] ** 2 + f["piye"] ** 2))
    assert np.all(np.abs(pp) <= e ** 2 + 3 * P ** 2)
    if Pi is not None:
        assert np.all(np.abs(Pi) <= P)
