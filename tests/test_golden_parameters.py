"""The defaults of the library, the oracle and the input generators against
the numbers the paper prints (tests/golden/paper_parameters.txt, each line
citing where the paper prints it)."""
import inspect
import os

import numpy as np
import pytest

import oracle
from paper_1802_04449_gb300 import clv
from paper_1802_04449_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        body, cite = line.split(";", 1)
        name, value = (s.strip() for s in body.split("="))
        assert cite.strip(), name           # every value says where the paper prints it
        out[name] = float(value)
    return out


G = golden()


def default(f, name):
    return inspect.signature(f).parameters[name].default


def test_every_golden_value_is_cited_and_used():
    assert set(G) == {"eps_cut_GeV_per_fm3", "tau_pi_coefficient", "gubser_lambda1_hat", "riemann_cs2",
                      "T_freezeout_GeV", "eta_w_PbPb_2760", "sigma_eta_PbPb_2760"}


def test_vacuum_cutoff_default():
    assert default(clv.Hydro.__init__, "eps_cut") == G["eps_cut_GeV_per_fm3"]
    assert default(oracle.Oracle.__init__, "eps_cut") == G["eps_cut_GeV_per_fm3"]


def test_relaxation_time_coefficient_default():
    # the oracle takes b explicitly; the library's 0 means the paper's b
    assert default(oracle.Oracle.__init__, "taupi_coef") == G["tau_pi_coefficient"]
    assert default(clv.Hydro.__init__, "taupi_coef") == 0.0
    assert I.HydroCase.__dataclass_fields__["taupi_coef"].default == 0.0


def test_gubser_second_order_setup():
    assert default(I.gubser_viscous, "lambda1_hat") == G["gubser_lambda1_hat"]
    assert default(I.gubser_viscous_case, "lambda1_hat") == G["gubser_lambda1_hat"]


def test_riemann_rarefaction_speed_of_sound():
    # the conformal EOS (eos=None) that the Riemann pins run with: P = eps/3, c_s^2 = 1/3
    o = oracle.Oracle(4, 1, 1, 0.1, 0.1, 0.1, 1.0, 0.01, eos=None)
    for e in (1e-3, 0.5, 10.0, 300.0):
        P, T, cs2 = o.eos(e)[:3]
        assert cs2 == pytest.approx(G["riemann_cs2"], rel=1e-15)
        assert P == pytest.approx(G["riemann_cs2"] * e, rel=1e-15)


def test_longitudinal_envelope_parameters():
    assert default(I.h_eta, "eta_w") == G["eta_w_PbPb_2760"]
    assert default(I.h_eta, "sigma_eta") == G["sigma_eta_PbPb_2760"]
    # Eq. (h_eta): 1 on the plateau |eta_s| <= eta_w, a half-Gaussian of width sigma_eta beyond
    w, s = G["eta_w_PbPb_2760"], G["sigma_eta_PbPb_2760"]
    assert I.h_eta(np.array([0.0, w, -w]), w, s) == pytest.approx([1.0, 1.0, 1.0])
    assert I.h_eta(w + s, w, s) == pytest.approx(np.exp(-0.5))
    assert I.h_eta(-(w + 2 * s), w, s) == pytest.approx(np.exp(-2.0))
