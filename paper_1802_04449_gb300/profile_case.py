"""Profiling driver: the 97x97x41 viscous hot-spot event evolved through the C
ABI, for capture under a profiler (the kernels of interest are the last
launches).  Usage:

    python -m paper_1802_04449_gb300.profile_case [--precision fp32|fp64]
        [--guess previous|cold|learned] [--skip S] [--steps K] [--no-autotune]
        [--surface] [--zeta-over-s Z] [--charge]

The tile shape is autotuned first (as bench.py does; its timing launches
come first), --skip S steps run next (reaching the later, more dilute
state), then K steps.  --guess learned trains the network briefly (FP64 states of another
seed of the same workload) before the run.  --surface then takes a slice,
runs 10 more steps, finds the freeze-out surface at T_f = 137 MeV between the
two slices (clv_fo_find) and computes the pi+, K+ and p spectra on the
41 x 15 x 48 grid from it (clv_cf_spectra): those launches come last.
--zeta-over-s Z > 0 evolves the bulk pressure too, --charge a smooth net
charge (their kernels run once per stage).
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--guess", default="previous", choices=["previous", "cold", "learned"])
    ap.add_argument("--skip", type=int, default=0)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--surface", action="store_true")
    ap.add_argument("--zeta-over-s", type=float, default=0.0)
    ap.add_argument("--charge", action="store_true")
    a = ap.parse_args(argv)

    import torch
    from paper_1802_04449_gb300 import clv
    from paper_1802_04449_gb300 import inputs as I
    from paper_1802_04449_gb300 import learned as L

    case = I.hotspot_event()
    prec = clv.CLV_FP32 if a.precision == "fp32" else clv.CLV_FP64
    params = None
    if a.guess == "learned":
        tc = I.hotspot_event(seed=1000)
        h = clv.from_case(tc, clv.CLV_FP64)
        h.set_initial(tc.eps, tc.ux, tc.uy, tc.ueta)
        X, Y = L.collect_samples(h, max(a.skip + a.steps, 40), 20).data()
        p, _ = L.train(X, Y, iters=1000, batch=32768, lr=2e-3, seed=7)
        params = p.cpu().numpy()
        h.close()
    g = clv.from_case(case, prec, zeta_over_s=a.zeta_over_s, charge=a.charge)
    g.set_initial(case.eps, case.ux, case.uy, case.ueta)
    if a.charge:
        import numpy as np
        g.set_initial_n(0.2 + 0.05 * np.cos(np.linspace(0.0, 6.283, case.eps.size)).reshape(case.eps.shape))
    if params is not None:
        g.set_mlp(params)
    g.set_guess({"previous": clv.CLV_GUESS_PREVIOUS, "cold": clv.CLV_GUESS_COLD,
                 "learned": clv.CLV_GUESS_MLP}[a.guess])
    if a.autotune:
        print("tile:", g.autotune(max_candidates=12, reps=3))
    if a.skip:
        g.step(a.skip)
    st = g.step(a.steps, stats=True)
    torch.cuda.synchronize()
    print("profile case done: tau %.3f, newton iters/solve %.3f, polished %d" %
          (st["tau"], st["n_newton_iters"] / max(1, st["n_newton_cells"]), st["n_polished"]))
    if a.surface:
        import numpy as np
        snap = g.fo_snapshot()
        g.step(10)
        eos = case.eos
        lne = eos["lne0"] + eos["dlne"] * np.arange(len(eos["T"]))
        eps_f = float(np.float32(np.exp(np.interp(0.137, eos["T"], lne))))
        finder = clv.FreezeoutFinder(g.fo_grid(), stream=g.stream)
        finder.find(snap, g.fo_current(), eps_f)
        Y, pT, _, phi, _ = I.spectra_grid()
        P_f = float(np.interp(np.log(eps_f), lne, eos["P"]))
        cf = clv.CooperFrye(["pi+", "K+", "p"], Y, pT, phi, 0.137, eps_f + P_f, True, prec, stream=g.stream)
        cf.spectra(finder.rec, d_nel=finder.count)
        _, _, n = finder.result()
        print("surface: %d elements at eps_f = %.4f" % (n, eps_f))


if __name__ == "__main__":
    main()
