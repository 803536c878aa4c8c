"""Meta-test: each pin must catch a plausible mistake.

The oracle is rebuilt with one deliberate mistake (compile-time PLANT=n, on
the CPU only) and at least one pin must then fail:
  1 I^{mu nu} sign flipped               -> transversality drift
  2 pi~ u~^tau/tau sign flipped           -> viscous Bjorken ODE
  3 S_T^tau sign flipped (as printed)     -> Bjorken power law
  4 eta flux divisor without tau          -> linearised eta wave
  5 transposed gradient in sigma          -> transversality drift
  6 Christoffel term of nabla_eta u^eta   -> transversality drift / Bjorken
  7 S_T^eta dropped                       -> linearised eta wave
  8 EOS argument E instead of E - M v     -> brute-force root solve (Gubser flow)
Freeze-out surface (clv_freezeout.c):
  9 normal along +grad eps                -> planar level set in time
 10 one tetrahedron of the prism dropped  -> coarea closed form per simplex
 11 Milne weight tau0 instead of the piece's tau -> planar level sets in space
 12 one simplex of the 24 left out        -> closed level set / planar in time
Cooper-Frye spectra (clv_cooperfrye.c):
 13 tau p^eta dSigma_eta multiplied by tau instead of divided -> particle number n u.dSigma
 14 quantum statistics sign flipped       -> Bessel closed form of the boost-invariant surface
 15 sign of the p~^eta u~^eta term of p.u -> particle number n u.dSigma
Net charge (clv_oracle.c, R19):
 16 the local-speed term of the charge flux with the wrong sign -> Gubser charge convergence
 17 initial N~^tau without the tau factor -> Bjorken n tau constant
Bulk pressure (clv_oracle.c, R20):
 18 the -Pi u~^tau/tau term of S_Pi dropped -> Bjorken bulk ODE
 19 sign of the zeta theta~ term flipped  -> Bjorken bulk ODE / sound wave
 20 root solve without the Pi pressure shift -> decomposition of T^{tau mu}
 21 Pi left out of the pressure in the T~ fluxes -> linearised sound wave
Velocity predictor (clv_oracle.c, R8 and the u* extrapolation of Sec. 3):
 22 first step without the pi-free step (u^{-1} = u^0) -> first-step predictor
 23 u^{n-1} never updated after a step    -> velocity history / second-order extrapolation
KT interface (clv_oracle.c, Sec. 3):
 24 right state reconstructed with the slope's sign flipped -> mirror symmetry (also Gubser, eta wave)
 25 right-side local speed from the left cell's c_s -> mirror symmetry (no other pin sees it)
Shear regulator (clv_oracle.c, R18):
 26 the cap's bound without its 3 P^2 term -> exact cap in a static box
 27 the ramp without its offset (eps/1e-3 instead of eps/1e-3 - 1) -> static-box ramp
Equation of state (clv_oracle.c, Sec. 3):
 28 table interpolation weights swapped for P -> numpy.interp on the nodes
 29 conformal T from eps with 90 in place of 30 -> Stefan-Boltzmann law
Initial state from T^{tau mu} (clv_oracle.c):
 30 T^{tau x} and T^{tau y} swapped on the way to the root solve -> perfect-fluid round trip
"""
import numpy as np
import pytest

import oracle
import test_oracle_flows as F
import test_oracle_bulk as BU
import test_oracle_charge as CH
import test_oracle_cooperfrye as CF
import test_oracle_freezeout as FO
import test_oracle_eos_prim as EP
import test_oracle_initial_T as IT
import test_oracle_predictor as PR
import test_oracle_symmetry as SY

CASES = {
    1: F.check_transversality,
    2: F.check_bjorken_viscous,
    3: F.check_bjorken_ideal,
    4: F.check_eta_wave,
    5: F.check_transversality,
    6: F.check_bjorken_viscous,
    7: F.check_eta_wave,
    8: F.check_gubser,
    9: FO.check_planar_tau,
    10: FO.check_simplices,
    11: FO.check_planar_axes,
    12: FO.check_closed_surface,
    13: CF.check_particle_number,
    14: CF.check_bjorken_bessel,
    15: CF.check_particle_number,
    16: CH.check_gubser_charge,
    17: CH.check_bjorken_charge,
    18: BU.check_bjorken_bulk,
    19: BU.check_bjorken_bulk,
    20: BU.check_decomposition,
    21: BU.check_bulk_sound_wave,
    22: PR.check_first_step_predictor,
    23: PR.check_velocity_history,
    24: SY.check_symmetries,
    25: SY.check_symmetries,
    26: F.check_regulator_cap_exact,
    27: F.check_regulator_ramp,
    28: EP.check_table_eos,
    29: EP.check_conformal_eos,
    30: IT.check_reproduce_T,
}


@pytest.mark.parametrize("plant", sorted(CASES))
def test_pin_catches_planted_mistake(plant):
    CASES[plant](plant=0)            # the correct oracle passes
    with pytest.raises(AssertionError):
        CASES[plant](plant=plant)    # the broken one fails
