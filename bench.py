#!/usr/bin/env python3
"""Benchmark: hydro cell-updates/s of one Heun step of (3+1)D viscous hydro
in Milne coordinates on GB300, through libclv's C ABI.

Workload (default): the viscous hot-spot event -- 97x97x41 cells, dx = dy =
d_eta = 0.2, dtau = 0.01 fm, tau0 = 0.4 fm, eta/s = 0.08, 2048 Gaussian hot
spots from Woods-Saxon thickness at b = 7 fm, synthetic crossover EOS table
(4096 nodes), zero initial velocity.  A step is one full Heun step (both
stages: KT fluxes, Milne and shear sources, pi update, primitive recovery)
over the grid; one cell-update is one cell advanced by one step.

value:  device-resident throughput of the FP32 path with the learned initial
        guess of the root solve (trained, untimed, on the FP64 solver's states
        of other seeds of the same workload); the FP64 path and the FP32 path
        with the previous-step and the cold-start guess are timed on the same grid
        beside it.  The state (~71 MB in FP32)
        fits in L2, so a 512 MiB buffer is written between timed steps
        (L2 flushed; the flush is outside the timed intervals).
e2e:    the same metric through the public API with host buffers: upload of
        the initial state from pinned memory, K steps, download of eps and u~.
With --gpus N (torchrun), each rank evolves its own event (seed + rank):
independent problems, no data-path collective, weak scaling.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "hydro cell-updates/s on GB300, FP32+learned vs FP64, % HBM roofline"
UNIT = "cell-updates/s"
# Algorithmic words moved per cell by each kernel of a step (each field once):
KERNEL_WORDS = {
    "stage1": 35,    # read T~ 4, pi~ 10, eps 1, u~ 3, u~^{n-1} 3; write T~' 4, pi~' 10
    "recover1": 15,  # read T~'^{tau mu} 4, pi~'^{tau mu} 4, u~ 3; write eps', u~' 4
    "stage2": 52,    # read T~' 4, pi~' 10, eps' 1, u~' 3, T~^n 4, pi~^n 10, u~^n 3, u~^{n-1} 3; write 14
    "recover2": 15,  # read T~^{tau mu} 4, pi~^{tau mu} 4, u~' 3; write eps, u~ 4
}
LEDGER_WORDS = 92    # the method's per-cell-update ledger for a fused step (each field once per stage)
KERNEL_READ_WORDS = {"stage1": 21, "recover1": 11, "stage2": 38, "recover2": 11}
# Words each FP32 kernel actually moves per cell (each field once): beyond
# the ledger, the stage kernels read the stored P and c_s of their input, and
# T~ is a float-float pair (the low parts of every T~ read and written); the
# recovery also writes P and c_s
KERNEL_MOVED_WORDS = {
    "stage1": 45,    # read T~ 4+4, pi~ 10, u~ 3, P, c_s, eps, u~^{n-1} 3; write T~' 4+4, pi~' 10
    "recover1": 21,  # read T~' 4+4, pi~'^{tau mu} 4, u~ 3; write eps', u~' 3, P', c_s'
    "stage2": 66,    # read T~' 8, pi~' 10, u~' 3, P', c_s', eps', T~^n 8, pi~^n 10, u~^n 3, u~^{n-1} 3; write 18
    "recover2": 21,
}
# Freeze-out surface finder (FP32): algorithmic bytes per hypercube (eps of
# both slices, each cell once) and per element (the 22-value record and its
# hypercube index written, u~ and pi~ of one cell of each slice read)
FO_BYTES_PER_CUBE = 2 * 4
FO_BYTES_PER_ELEMENT = 22 * 4 + 8 + 2 * 13 * 4
# Cooper-Frye sum: flops of one (element, momentum) pair with delta f, an FMA
# counted as 2 and exp2 / reciprocal as 1 each.  What depends on the element
# and (Y, pT) only is formed once for the 8 phi points of a thread: e^(Y-eta),
# cosh, sinh 8, p^tau and tau p^eta 2, their parts of p.dSigma and p.u 6, of
# p p pi 14 -> 30 / 8 = 3.75 per pair; per phi point: p.dSigma 4, p.u 4,
# exponent 2, exp2 1, f 2, p p pi 10, (1 - s f) q + 1 4, product and sum 3 -> 30
CF_FLOPS_PER_PAIR = 33.75
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# algorithmic words per cell of one launch of the optional kernels: bulk reads
# eps, u~ (3), c_s and Pi of the stage's input, Pi^n, u~^n (3) and u~^{n-1} (3),
# writes Pi (15); charge reads N~ of the stage's input, u~ (3), c_s and N~^n,
# writes N~ (7)
BULK_WORDS = 15
CHARGE_WORDS = 7
HBM_NOMINAL_GBS = 7900.0   # GB300 HBM3e, nominal (context beside the measured copy peak)
KERNEL_NAMES = {"stage1": "stage_tile_kernel<float,1,viscous>", "recover1": "recover_kernel<float,viscous>",
                "stage2": "stage_tile_kernel<float,2,viscous>", "recover2": "recover_kernel<float,viscous>"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload(seed_offset=0):
    from paper_1802_04449_gb300 import inputs as I
    return I.hotspot_event(seed=12345 + seed_offset)


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_1802_04449_gb300 import build as B
    from paper_1802_04449_gb300 import clv
    from paper_1802_04449_gb300 import learned as L

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    B.build()
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    case = workload(rank)
    N = case.ncells
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def barrier():
        if ws > 1:
            dist.barrier()

    def timed_run(precision, steps, warmup, kernel_timing=False, params=None, guess=None, ev=None, flush_l2=True,
                  n0=None, **hkw):
        ev = case if ev is None else ev
        g = clv.from_case(ev, precision, **hkw)
        g.set_initial_case(ev)
        if n0 is not None:
            g.set_initial_n(n0)
        if params is not None:
            g.set_mlp(params)
            g.set_guess(clv.CLV_GUESS_MLP)
        elif guess is not None:
            g.set_guess(guess)
        tile = g.autotune(max_candidates=12, reps=3) if args.autotune else g.tile()
        g.step(warmup)
        torch.cuda.synchronize()
        g.enable_kernel_timing(kernel_timing)
        stream = g.stream
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        torch.cuda.synchronize()
        for i in range(steps):
            if flush_l2:
                flush.fill_(i & 0xFF)                # evict the state from L2 (not timed)
            evs[i][0].record(stream)
            g.step(1)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        kt = g.kernel_times() if kernel_timing else None
        try:
            st = g.stats()
        except clv.ClvError as e:          # reported in the JSON line, not hidden
            st = {"error": str(e)}
        g.close()
        st["tile"] = tile
        return ms, kt, st

    # ---- the learned guess (setup, not timed): states of the FP64 solver on
    # other seeds of the same workload, every train_every steps over the timed
    # span, then Adam on the GPU
    t_setup = time.perf_counter()
    buf = None
    for k in range(args.train_events):
        tc = workload(1000 + 97 * k + rank)
        h = clv.from_case(tc, clv.CLV_FP64)
        h.set_initial(tc.eps, tc.ux, tc.uy, tc.ueta)
        if buf is None:
            buf = L.SampleBuffer(torch, dev, args.train_events * (args.steps // args.train_every + 1) * tc.ncells)
        L.collect_samples(h, args.steps, args.train_every, buf)
        h.close()
    Xs, Ys = buf.data()
    params, losses = L.train(Xs, Ys, iters=args.train_iters, batch=32768, lr=2e-3, seed=7)
    losses = losses.cpu().numpy()
    params_host = params.cpu().numpy()
    learned = {"samples": int(Xs.shape[0]), "events": args.train_events, "every": args.train_every,
               "adam_iters": args.train_iters, "batch": 32768,
               "loss_first10": float(losses[:10].mean()), "loss_last100": float(losses[-100:].mean()),
               "setup_s": time.perf_counter() - t_setup}
    del buf, Xs, Ys, params

    # ---- FP32 + learned guess: the headline value, with per-kernel event timing.
    # nvidia-smi samples the clocks from here through the last timed
    # configuration below (it needs a moment to start; the headline alone
    # lasts a fraction of a second)
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.5)
    ms32, kt, st32 = timed_run(clv.CLV_FP32, args.steps, args.warmup, kernel_timing=True, params=params_host)
    # ---- FP32 with the previous-step guess, and the FP64 path (fewer steps:
    # it is ALU-bound), on the same grid
    ms32p, _, st32p = timed_run(clv.CLV_FP32, args.steps, args.warmup)
    ms32c, _, st32c = timed_run(clv.CLV_FP32, args.steps, args.warmup, guess=clv.CLV_GUESS_COLD)
    steps64 = max(3, args.steps // 4)
    ms64, _, st64 = timed_run(clv.CLV_FP64, steps64, args.warmup)

    t_local = torch.tensor([ms32, ms32p, ms32c, ms64], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
    ms32_max, ms32p_max, ms32c_max, ms64_max = t_local.tolist()
    value = ws * N * args.steps / (ms32_max / 1e3)
    value32p = ws * N * args.steps / (ms32p_max / 1e3)
    value32c = ws * N * args.steps / (ms32c_max / 1e3)
    value64 = ws * N * steps64 / (ms64_max / 1e3)

    # FMA rates of this GPU (the ALU-roofline peaks), measured after the
    # timed runs above
    fma64 = clv.fma_rate(clv.CLV_FP64)
    fma32 = clv.fma_rate(clv.CLV_FP32)
    f64_flops = load_fp64_flops()

    def per(a, b):
        return (a / b) if (a is not None and b) else None

    for name, st in (("learned", st32), ("previous", st32p), ("cold", st32c)):
        learned[f"newton_iters_per_solve_{name}"] = per(st.get("n_newton_iters"), st.get("n_newton_cells"))
        learned[f"warp_max_iters_per_warp_{name}"] = per(st.get("n_newton_warp_max"), st.get("n_newton_warps"))
        learned[f"polish_iters_per_polished_{name}"] = per(st.get("n_polish_iters"), st.get("n_polished"))

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (case.eps, case.ux, case.uy, case.ueta)]
        out = torch.empty((4, N), dtype=torch.float64).pin_memory()
        g = clv.from_case(case, clv.CLV_FP32)
        host_in = [p.numpy() for p in pinned]
        g.set_initial(*host_in)                      # warm-up
        g.set_mlp(params_host)
        g.set_guess(clv.CLV_GUESS_MLP)
        if args.autotune:
            g.autotune(max_candidates=12, reps=3)
        g.step(args.warmup)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        g.set_mlp(params_host)
        g.set_initial(*host_in)
        try:
            g.step(args.steps, stats=True)
        except clv.ClvError as e:
            print(f"e2e run reported: {e}", file=sys.stderr)
        g.get(["eps", "ux", "uy", "ueta"], out=out.numpy())
        t1 = time.perf_counter()
        g.close()
        et = torch.tensor([t1 - t0], dtype=torch.float64, device=dev)
        if ws > 1:
            dist.all_reduce(et, op=dist.ReduceOp.MAX)
        e2e = {"value": ws * N * args.steps / et.item(), "unit": UNIT,
               "h2d_bytes_per_step": 4 * N * 8 / args.steps,
               "d2h_bytes_per_step": (4 * N * 8 + 64) / args.steps,
               "includes": "H2D of the network (20 KB) and of the initial state (pinned), the first-step "
                           f"ideal predictor, {args.steps} steps, stats read-back, D2H of eps and u~"}

    # ---- roofline of the dominant kernel, from live per-kernel event timing
    peak, peak_kind = measured_peaks()
    word = 4
    avg_ms = {k: (ms / n if n else 0.0) for k, (ms, n) in kt.items()}
    tot_ms = {k: ms for k, (ms, n) in kt.items()}
    dom = max(tot_ms, key=tot_ms.get)
    alg = KERNEL_WORDS[dom] * word * N
    achieved = alg / (avg_ms[dom] / 1e3) / 1e9
    tr = load_traffic(dom, st32.get("tile") if dom.startswith("stage") else None)
    roof = {"bound": "hbm", "kernel": KERNEL_NAMES[dom], "achieved": achieved,
            "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
            "nominal_peak": HBM_NOMINAL_GBS, "frac_of_nominal": achieved / HBM_NOMINAL_GBS,
            "traffic": (tr[0] + tr[1]) if tr else None,
            "read_traffic_ratio": (tr[0] / (KERNEL_READ_WORDS[dom] * word * N)) if tr else None,
            "l2_resident": "the 71 MB FP32 state of this event stays in L2 within a step (L2 is flushed "
                           "between steps); the HBM-bound fractions are those of the large event and the batch "
                           "(hbm_resident_frac)",
            "algorithmic_bytes_per_launch": alg,
            "moved_bytes_per_launch": KERNEL_MOVED_WORDS[dom] * word * N,
            "kernel_ms_avg": avg_ms,
            "kernel_share": {k: v / sum(tot_ms.values()) for k, v in tot_ms.items()},
            "ledger_bytes_per_cell_update": LEDGER_WORDS * word,
            "step_frac_of_peak": (value / ws) * LEDGER_WORDS * word / 1e9 / peak}

    # ---- the large single event with mini-jet initial flow (261x261x121,
    # 8.2M cells; its ~1.5 GB FP32 state is far larger than L2, so no flush is
    # needed): FP32 + learned guess (the network above) vs FP64, fewer steps
    large = None
    if args.large:
        from paper_1802_04449_gb300 import inputs as I
        lc = I.minijet_event(seed=2024 + rank)
        NL = lc.ncells
        sL = max(3, args.steps // 10)
        msL, ktL, stL = timed_run(clv.CLV_FP32, sL, 3, kernel_timing=True, params=params_host, ev=lc, flush_l2=False)
        sL64 = max(2, sL // 5)
        msL64, _, stL64 = timed_run(clv.CLV_FP64, sL64, 2, ev=lc, flush_l2=False)
        tl = torch.tensor([msL, msL64], dtype=torch.float64, device=dev)
        if ws > 1:
            dist.all_reduce(tl, op=dist.ReduceOp.MAX)
        msL_max, msL64_max = tl.tolist()
        avgL = {k: (ms / n if n else 0.0) for k, (ms, n) in ktL.items()}
        domL = max(avgL, key=avgL.get)
        achL = KERNEL_WORDS[domL] * 4 * NL / (avgL[domL] / 1e3) / 1e9
        trL = load_traffic("large_" + domL, stL.get("tile") if domL.startswith("stage") else None)
        valL = ws * NL * sL / (msL_max / 1e3)
        large = {"workload": "hot-spot event with mini-jet initial flow 261x261x121, dx=dy=0.08, deta=0.1, "
                             "dtau=0.005 fm, eta/s=0.16, 8000 spots (p_T exponential, mean 1.5 GeV), "
                             "crossover EOS table 4096",
                 "cells_per_event": NL, "steps": sL, "l2": "state (1.5 GB FP32) far larger than L2; no flush",
                 "value": valL, "unit": UNIT, "ms_per_step": msL_max / sL,
                 "fp64": {"value": ws * NL * sL64 / (msL64_max / 1e3), "steps": sL64,
                          "ms_per_step": msL64_max / sL64},
                 "roofline": {"bound": "hbm", "kernel": KERNEL_NAMES[domL], "achieved": achL, "peak": peak,
                              "unit": "GB/s", "frac": achL / peak, "kernel_ms_avg": avgL,
                              "traffic": (trL[0] + trL[1]) if trL else None,
                              "read_traffic_ratio": (trL[0] / (KERNEL_READ_WORDS[domL] * 4 * NL)) if trL else None,
                              "algorithmic_bytes_per_launch": KERNEL_WORDS[domL] * 4 * NL,
                              "moved_bytes_per_launch": KERNEL_MOVED_WORDS[domL] * 4 * NL,
                              "step_frac_of_peak": (valL / ws) * LEDGER_WORDS * 4 / 1e9 / peak},
                 "newton_iters_per_solve": per(stL.get("n_newton_iters"), stL.get("n_newton_cells")),
                 "stats_fp32": {k: stL.get(k) for k in ("tau", "eps_max", "T_max", "n_polished", "n_rootfail",
                                                        "error_word", "error", "tile")},
                 "stats_fp64": {k: stL64.get(k) for k in ("tau", "eps_max", "n_rootfail", "error_word", "error",
                                                          "tile")}}

    # ---- the large event over its whole lifetime (tau0 until max T < 137
    # MeV, the paper's stopping temperature): FP32 + learned guess, the
    # stopping rule read every CHUNK steps from the device reduction, timed
    # as a whole with events; then the FP64 path over the same number of
    # steps, and eps of the two compared at the end
    lifetime = None
    if args.lifetime:
        from paper_1802_04449_gb300 import inputs as I
        lc = I.minijet_event(seed=2024 + rank)
        T_F, CHUNK, MAXSTEPS = 0.137, 50, 2400

        def run_life(prec, nsteps=None):
            g = clv.from_case(lc, prec)
            g.set_initial_case(lc)
            if prec == clv.CLV_FP32:
                g.set_mlp(params_host)
                g.set_guess(clv.CLV_GUESS_MLP)
            if args.autotune:
                g.autotune(max_candidates=12, reps=3)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(g.stream)
            done, st, err = 0, None, None
            while done < (nsteps or MAXSTEPS):
                k = CHUNK if nsteps is None else min(CHUNK, nsteps - done)
                try:
                    st = g.step(k, stats=True)
                except clv.ClvError as e:   # reported in the JSON line, not hidden
                    err = str(e)
                    break
                done += k
                if nsteps is None and st["T_max"] < T_F:
                    break
            e1.record(g.stream)
            torch.cuda.synchronize()
            eps = g.get(["eps"])["eps"]
            g.close()
            return done, e0.elapsed_time(e1), st, err, eps

        n32, ms_l32, st_l32, err32, eps32 = run_life(clv.CLV_FP32)
        n64, ms_l64, st_l64, err64, eps64 = run_life(clv.CLV_FP64, n32)
        live = eps64 > 1e-3
        rel = np.zeros_like(eps64)
        rel[live] = np.abs(eps32[live] / eps64[live] - 1)
        imax = np.unravel_index(int(np.argmax(rel)), rel.shape)
        edge = min(min(i, n - 1 - i) for i, n in zip(imax, rel.shape))
        dense = eps64 > 0.1
        lifetime = {
            "workload": "the 261x261x121 mini-jet event from tau0 = 0.4 fm until max T < 137 MeV",
            "steps": n32, "tau_end": st_l32["tau"] if st_l32 else None,
            "T_max_end": st_l32["T_max"] if st_l32 else None,
            "value": ws * lc.ncells * n32 / (ms_l32 / 1e3), "unit": UNIT, "seconds": ms_l32 / 1e3,
            "stopping_rule": f"T_max from the device reduction every {CHUNK} steps (a stats step)",
            "error_word": st_l32["error_word"] if st_l32 else None, "error": err32,
            "n_rootfail": st_l32["n_rootfail"] if st_l32 else None,
            "fp64": {"steps": n64, "value": ws * lc.ncells * n64 / (ms_l64 / 1e3), "seconds": ms_l64 / 1e3,
                     "error_word": st_l64["error_word"] if st_l64 else None, "error": err64},
            "accuracy_vs_fp64": {"cells_compared": int(live.sum()),
                                 "eps_linf_rel_where_eps_gt_1e-3":
                                     float(np.max(np.abs(eps32[live] / eps64[live] - 1))) if live.any() else None,
                                 "eps_l1_rel": float(np.abs(eps32 - eps64).sum() / np.abs(eps64).sum()),
                                 "eps_linf_rel_where_eps_gt_0.1": float(rel[dense].max()) if dense.any() else None,
                                 "worst_cell": {"index": [int(i) for i in imax], "eps_fp64": float(eps64[imax]),
                                                "cells_from_grid_edge": int(edge)},
                                 "cells_over_1e-4": int((rel > 1e-4).sum()),
                                 "by_eps_band": {f"[{lo:g},{hi:g})": {
                                     "cells": int(((eps64 >= lo) & (eps64 < hi)).sum()),
                                     "linf": float(rel[(eps64 >= lo) & (eps64 < hi)].max())
                                     if ((eps64 >= lo) & (eps64 < hi)).any() else None,
                                     "over_1e-4": int((rel[(eps64 >= lo) & (eps64 < hi)] > 1e-4).sum())}
                                     for lo, hi in ((1e-3, 2e-3), (2e-3, 1e-2), (1e-2, 0.1), (0.1, 1e9))}},
        }
        del eps32, eps64

    # ---- freeze-out surface of the same event: T_f = 137 MeV (the paper's
    # stopping temperature) through the EOS table, between the slices at
    # tau = 2.4 and 2.5 fm; the four launches of clv_fo_find timed with
    # events on the handle's stream, L2 flushed between calls (untimed)
    freezeout = cooperfrye = None
    if args.freezeout:
        from paper_1802_04449_gb300 import inputs as I
        g = clv.from_case(case, clv.CLV_FP32)
        g.set_initial_case(case)
        g.set_mlp(params_host)
        g.set_guess(clv.CLV_GUESS_MLP)
        g.step(200)
        snap = g.fo_snapshot()
        g.step(10)
        cur = g.fo_current()
        eos = case.eos
        lne = eos["lne0"] + eos["dlne"] * np.arange(len(eos["T"]))
        eps_f = float(np.float32(np.exp(np.interp(0.137, eos["T"], lne))))
        finder = clv.FreezeoutFinder(g.fo_grid(), device=dev, stream=g.stream)
        for _ in range(3):
            finder.find(snap, cur, eps_f)
        reps = 50
        fev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        torch.cuda.synchronize()
        for i in range(reps):
            flush.fill_(i & 0xFF)
            fev[i][0].record(g.stream)
            finder.find(snap, cur, eps_f)
            fev[i][1].record(g.stream)
        torch.cuda.synchronize()
        fms = sum(a.elapsed_time(b) for a, b in fev) / reps
        _, _, nel = finder.result()
        gr = g.fo_grid()
        ncube = (gr.nx - 1) * (gr.ny - 1) * (gr.neta - 1)
        fo_alg = FO_BYTES_PER_CUBE * ncube + FO_BYTES_PER_ELEMENT * nel
        fo_ach = fo_alg / (fms / 1e3) / 1e9
        # ---- smooth Cooper-Frye spectra of pi+, K+ and p on the paper's
        # 41 x 15 x 48 grid over that surface, straight from the finder's
        # device records and count (ALU-bound: FP32 lanes)
        Yg, pTg, _, phig, _ = I.spectra_grid()
        lne_P = np.interp(np.log(eps_f), lne, eos["P"])
        cf = clv.CooperFrye(["pi+", "K+", "p"], Yg, pTg, phig, 0.137, eps_f + float(lne_P), True, clv.CLV_FP32,
                            device=dev, stream=g.stream)
        for _ in range(3):
            cf.spectra(finder.rec, d_nel=finder.count)
        creps = 20
        cev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(creps)]
        torch.cuda.synchronize()
        for i in range(creps):
            flush.fill_(i & 0xFF)
            cev[i][0].record(g.stream)
            cf.spectra(finder.rec, d_nel=finder.count)
            cev[i][1].record(g.stream)
        torch.cuda.synchronize()
        cms = sum(a.elapsed_time(b) for a, b in cev) / creps
        pairs = 3 * nel * len(Yg) * len(pTg) * len(phig)
        cf_ach = CF_FLOPS_PER_PAIR * pairs / (cms / 1e3) / 1e12
        cooperfrye = {"workload": f"pi+, K+, p on 41 x 15 x 48 (Y, pT, phi) points over the {nel} elements above, "
                                  "delta f on", "ms_per_call": cms, "pairs": pairs,
                      "value": pairs / (cms / 1e3), "unit": "element-momentum pairs/s", "launches_per_call": 3,
                      "l2": "flushed between calls (512 MiB write, untimed)",
                      "roofline": {"bound": "alu", "kernel": "cf_sum_kernel<float, viscous>",
                                   "achieved": cf_ach, "peak": FP32_ALU_TFLOPS, "unit": "TFLOP/s",
                                   "frac": cf_ach / FP32_ALU_TFLOPS, "flops_per_pair": CF_FLOPS_PER_PAIR,
                                   "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz",
                                   "frac_of_measured_fma_rate": cf_ach / fma32}}
        freezeout = {"workload": "the same event at tau = 2.4 -> 2.5 fm (10 steps apart), T_f = 137 MeV",
                     "eps_f": eps_f, "hypercubes": ncube, "elements": nel, "ms_per_find": fms,
                     "value": ncube / (fms / 1e3), "unit": "hypercubes/s", "launches_per_find": 4,
                     "l2": "flushed between calls (512 MiB write, untimed)",
                     "roofline": {"bound": "hbm", "kernel": "clv_fo_find (classify, scan, compact, elements)",
                                  "achieved": fo_ach, "peak": peak, "unit": "GB/s", "frac": fo_ach / peak,
                                  "algorithmic_bytes_per_find": fo_alg}}
        g.close()

    # ---- event-by-event batch: uneven grids in one handle, one persistent
    # stage launch per stage (state ~19 GB FP32, far larger than L2)
    batch = None
    if args.batch_events > 0:
        from paper_1802_04449_gb300 import inputs as I
        evs = I.batch_events(args.batch_events, seed0=1000 + 100000 * rank)
        NB = sum(e.ncells for e in evs)

        def timed_batch(prec, steps, warmup, params=None):
            bt = clv.Batch(evs, prec)
            for k, e in enumerate(evs):
                bt.set_event(k, e.eps, e.ux, e.uy, e.ueta)
            if params is not None:
                bt.set_mlp(params)
                bt.set_guess(clv.CLV_GUESS_MLP)
            bt.step(warmup)
            tuned = bt.autotune(max_candidates=8, reps=2)   # tiling policy of the batch (untimed setup)
            torch.cuda.synchronize()
            bt.enable_kernel_timing(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            torch.cuda.synchronize()
            e0.record(bt.stream)
            bt.step(steps)
            e1.record(bt.stream)
            torch.cuda.synchronize()
            barrier()
            kt = bt.kernel_times()
            try:
                st = bt.stats()
            except clv.ClvError as ex:
                st = {"error": str(ex)}
            bt.close()
            return e0.elapsed_time(e1), kt, st, tuned

        sB = max(3, args.steps // 8)
        msB, ktB, stB, tunedB = timed_batch(clv.CLV_FP32, sB, 2, params_host)
        sB64 = max(2, sB // 10)
        msB64, _, stB64, tunedB64 = timed_batch(clv.CLV_FP64, sB64, 1)
        tb = torch.tensor([msB, msB64], dtype=torch.float64, device=dev)
        if ws > 1:
            dist.all_reduce(tb, op=dist.ReduceOp.MAX)
        msB_max, msB64_max = tb.tolist()
        avgB = {k: (ms / n if n else 0.0) for k, (ms, n) in ktB.items()}
        domB = max(avgB, key=avgB.get)
        achB = KERNEL_WORDS[domB] * 4 * NB / (avgB[domB] / 1e3) / 1e9
        valB = ws * NB * sB / (msB_max / 1e3)
        batch = {"workload": f"{len(evs)} events, nx = ny odd in [65, 129], neta odd in [21, 61], dx in "
                             "[0.15, 0.3] fm (deta = dx), b in [0, 12] fm, eta/s in {0, 0.08, 0.16}, "
                             "hot spots scaled by N_bin(b), crossover EOS table 4096",
                 "events": len(evs), "cells": NB, "steps": sB, "value": valB, "unit": UNIT,
                 "ms_per_step": msB_max / sB, "launch": "one persistent stage launch per stage (a CTA per SM, "
                                                          "work items most expensive first) + one root-solve launch",
                 "schedule": {"fp32": {"max_threads": tunedB["TJ"], "chunk_planes": tunedB["CX"],
                                       "stage1_ms": tunedB["ms"]},
                              "fp64": {"max_threads": tunedB64["TJ"], "chunk_planes": tunedB64["CX"],
                                       "stage1_ms": tunedB64["ms"]},
                              "how": "clv_autotune on the started batch: thread cap x x-chunk policies, "
                                     "stage-1 launches timed, untimed setup"},
                 "fp64": {"value": ws * NB * sB64 / (msB64_max / 1e3), "steps": sB64,
                          "ms_per_step": msB64_max / sB64},
                 "roofline": {"bound": "hbm", "kernel": KERNEL_NAMES[domB].replace("stage_tile_kernel",
                                                                                   "stage_batch_kernel"),
                              "achieved": achB, "peak": peak, "unit": "GB/s", "frac": achB / peak,
                              "kernel_ms_avg": avgB,
                              "step_frac_of_peak": (valB / ws) * LEDGER_WORDS * 4 / 1e9 / peak},
                 "newton_iters_per_solve": per(stB.get("n_newton_iters"), stB.get("n_newton_cells")),
                 "stats_fp32": {k: stB.get(k) for k in ("tau", "eps_max", "n_polished", "n_rootfail", "error_word",
                                                        "error")},
                 "stats_fp64": {k: stB64.get(k) for k in ("tau", "eps_max", "n_rootfail", "error_word", "error")}}
        del evs

    # ---- the optional fields on the headline event (FP32 + learned guess):
    # bulk pressure (zeta/s = 0.1) and net charge.  Their kernels run inside the
    # stage-kernel timing slots (bulk: both stages; charge: stage 1 in slot 2,
    # stage 2 in none), so each kernel's time is the slot's growth over the
    # headline run, and its bandwidth the algorithmic bytes over that time
    options = None
    if args.options:
        so = max(20, args.steps // 4)
        msBk, ktBk, stBk = timed_run(clv.CLV_FP32, so, args.warmup, kernel_timing=True, params=params_host,
                                     zeta_over_s=0.1)
        n0 = 0.2 + 0.05 * np.cos(np.linspace(0.0, 6.283, N)).reshape(case.eps.shape)
        msCh, ktCh, stCh = timed_run(clv.CLV_FP32, so, args.warmup, kernel_timing=True, params=params_host,
                                     charge=True, n0=n0)
        avg = lambda kt_: {k: (ms / n if n else 0.0) for k, (ms, n) in kt_.items()}
        a0, aB, aC = avg(kt), avg(ktBk), avg(ktCh)
        t_bulk = 0.5 * ((aB["stage1"] - a0["stage1"]) + (aB["stage2"] - a0["stage2"]))
        t_charge = aC["stage2"] - a0["stage2"]
        ach_b = BULK_WORDS * 4 * N / (t_bulk / 1e3) / 1e9 if t_bulk > 0 else None
        ach_c = CHARGE_WORDS * 4 * N / (t_charge / 1e3) / 1e9 if t_charge > 0 else None
        options = {"workload": "the headline event, FP32 + learned guess, L2 flushed between steps",
                   "steps": so,
                   "bulk": {"zeta_over_s": 0.1, "value": N * so / (msBk / 1e3), "unit": UNIT,
                            "ms_per_step": msBk / so, "step_overhead": (msBk / so) / (ms32 / args.steps) - 1.0,
                            "launches_per_step": 7,
                            "roofline": {"bound": "hbm", "kernel": "bulk_stage_kernel<float>", "ms_avg": t_bulk,
                                         "achieved": ach_b, "peak": peak, "unit": "GB/s",
                                         "frac": (ach_b / peak) if ach_b else None,
                                         "algorithmic_bytes_per_launch": BULK_WORDS * 4 * N},
                            "error_word": stBk.get("error_word")},
                   "charge": {"value": N * so / (msCh / 1e3), "unit": UNIT, "ms_per_step": msCh / so,
                              "step_overhead": (msCh / so) / (ms32 / args.steps) - 1.0, "launches_per_step": 7,
                              "roofline": {"bound": "hbm", "kernel": "charge_stage_kernel<float>", "ms_avg": t_charge,
                                           "achieved": ach_c, "peak": peak, "unit": "GB/s",
                                           "frac": (ach_c / peak) if ach_c else None,
                                           "algorithmic_bytes_per_launch": CHARGE_WORDS * 4 * N},
                              "error_word": stCh.get("error_word")}}

    clocks = sampler.stop()
    clocks["covers"] = ("from the headline through the batch: every timed configuration, e2e, freeze-out, "
                        "Cooper-Frye and the bulk and charge runs included")

    # ---- accuracy of the FP32 + learned-guess path on the headline event,
    # against the FP64 GPU path on the same grid (which the parity tests hold
    # to 1e-10 of the FP64 oracle): at the parity tests' 40-step horizon and
    # at the end of the headline run's span (warm-up + timed steps); untimed
    accuracy = None
    if args.accuracy:
        span = args.warmup + args.steps
        g32 = clv.from_case(case, clv.CLV_FP32)
        g32.set_initial_case(case)
        g32.set_mlp(params_host)
        g32.set_guess(clv.CLV_GUESS_MLP)
        g64 = clv.from_case(case, clv.CLV_FP64)
        g64.set_initial_case(case)
        marks, done = sorted({min(40, span), span}), 0
        acc = {}
        for m in marks:
            g32.step(m - done)
            g64.step(m - done)
            done = m
            e32, e64 = g32.get(["eps"])["eps"], g64.get(["eps"])["eps"]
            live = e64 > 1e-3
            acc[str(m)] = {"tau": g64.time()[0], "cells_compared": int(live.sum()),
                           "eps_linf_rel_where_eps_gt_1e-3": float(np.max(np.abs(e32[live] / e64[live] - 1))),
                           "eps_l1_rel": float(np.abs(e32 - e64).sum() / np.abs(e64).sum())}
        # on to the event's end (max T < 137 MeV, read every 20 steps): the
        # error by density band
        while done < 4000:
            st = g32.step(20, stats=True)
            g64.step(20)
            done += 20
            if st["T_max"] < 0.137:
                break
        e32, e64 = g32.get(["eps"])["eps"], g64.get(["eps"])["eps"]
        rel = np.zeros_like(e64)
        live = e64 > 1e-3
        rel[live] = np.abs(e32[live] / e64[live] - 1)
        bands = {}
        for lo, hi in ((1e-3, 2e-3), (2e-3, 1e-2), (1e-2, 0.1), (0.1, 1e9)):
            b = (e64 >= lo) & (e64 < hi)
            bands[f"[{lo:g},{hi:g})"] = {"cells": int(b.sum()), "linf": float(rel[b].max()) if b.any() else None,
                                         "over_1e-4": int((rel[b] > 1e-4).sum())}
        acc["to_T_max_below_137_MeV"] = {"steps": done, "tau": g64.time()[0], "cells_compared": int(live.sum()),
                                         "eps_linf_rel_where_eps_gt_1e-3": float(rel.max()),
                                         "eps_l1_rel": float(np.abs(e32 - e64).sum() / np.abs(e64).sum()),
                                         "by_eps_band": bands}
        g32.close()
        g64.close()
        accuracy = {"vs": "the FP64 GPU path on the same grid (held to 1e-10 of the FP64 oracle by the parity tests)",
                    "after_steps": acc}

    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "viscous hot-spot event 97x97x41, eta/s=0.08, crossover EOS table 4096, "
                               "2048 spots, b=7 fm, dtau=0.01 fm",
                   "cells_per_event": N, "events_per_gpu": 1,
                   "precision": "fp32 stencil and root solve from the learned guess (bf16 tensor-core MLP, "
                                "fp32 accumulate); fp64 root refinement at v > 0.999 and near the vacuum cut; "
                                "fp64 reductions",
                   "l2": "flushed between timed steps (512 MiB write, untimed)",
                   "parallelism": f"independent events, {ws} rank(s)"},
        "fp64": {"value": value64, "unit": UNIT, "steps": steps64, "ms_per_step": ms64_max / steps64,
                 "roofline": {"bound": "alu", "kernel": "FP64 step (stage and recovery kernels)",
                              "achieved": (f64_flops * value64 / ws / 1e12) if f64_flops else None,
                              "peak": fma64, "unit": "TFLOP/s",
                              "frac": (f64_flops * value64 / ws / 1e12 / fma64) if f64_flops else None,
                              "flops_per_cell_update": f64_flops,
                              "peak_kind": "measured: clv_fma_rate, independent FP64 FMA chains on every SM",
                              "hbm_frac": value64 / ws * LEDGER_WORDS * 8 / 1e9 / peak}},
        "alu_peaks_tflops": {"fp64_measured": fma64, "fp32_measured": fma32, "fp32_derived": FP32_ALU_TFLOPS},
        "fp32_previous_guess": {"value": value32p, "unit": UNIT, "steps": args.steps,
                                "ms_per_step": ms32p_max / args.steps},
        "fp32_cold_guess": {"value": value32c, "unit": UNIT, "steps": args.steps,
                            "ms_per_step": ms32c_max / args.steps},
        "learned_guess": learned,
        "accuracy": accuracy,
        "options": options,
        "large_event": large,
        "large_event_lifetime": lifetime,
        "batch": batch,
        "freezeout": freezeout,
        "cooperfrye": cooperfrye,
        "roofline": roof,
        "e2e": e2e,
        # per step: two stages of (stage kernel, root solve) and the tau advance
        "gpu_launches": 5 * args.steps,
        "clocks": clocks,
        "stats_fp32": {k: st32.get(k) for k in ("tau", "eps_max", "T_max", "E_tot", "n_polished", "n_rootfail",
                                                "n_fp32_nonconverged", "error_word", "error", "tile")},
        "stats_fp64": {k: st64.get(k) for k in ("tau", "eps_max", "E_tot", "n_rootfail", "error_word", "error",
                                                "tile")},
    }
    roof["hbm_resident_frac"] = {"large_event": large["roofline"]["frac"] if large else None,
                                 "batch": batch["roofline"]["frac"] if batch else None}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(res))
    if ws > 1:
        dist.destroy_process_group()


def load_traffic(dom, tile):
    """DRAM bytes per launch of kernel slot ``dom`` from the committed ncu
    summary: lines ``traffic <slot> <read bytes> <write bytes>
    <kernel-source-hash> <TJxTKxCX>`` in profiles/traffic.txt.  Returns
    (read, write), or None when absent, when the kernel sources changed since
    the counters were taken, or (stage slots) when the run used another tile
    shape."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    want = kernel_source_hash()
    shape = f"{tile['TJ']}x{tile['TK']}x{tile['CX']}" if tile else "-"
    with open(p) as f:
        for line in f:
            parts = line.split()
            if (len(parts) == 6 and parts[0] == "traffic" and parts[1] == dom and parts[4] == want
                    and (parts[5] == "-" or parts[5] == shape)):
                return float(parts[2]), float(parts[3])
    return None


def load_fp64_flops():
    """FP64 flops per cell-update of the FP64 step (an FMA counts as 2) from
    the ncu instruction counts in profiles/fp64_flops.txt (a line ``flops
    <per cell-update> <kernel-source-hash>``); None once the kernels changed."""
    p = os.path.join(ROOT, "profiles", "fp64_flops.txt")
    if not os.path.exists(p):
        return None
    want = kernel_source_hash()
    with open(p) as f:
        for line in f:
            parts = line.split()
            if len(parts) == 3 and parts[0] == "flops" and parts[2] == want:
                return float(parts[1])
    return None


def kernel_source_hash():
    """Hash of the device-code headers that define the stage and recovery
    kernels (host-side API changes leave it unchanged)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1802_04449_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith(".cuh"):
            with open(os.path.join(csrc, fn), "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:16]


def cpu_baseline(budget_s):
    """The FP64 oracle as it stands, all host cores, bounded sample of the
    same workload: as many steps as fit in ~budget_s seconds (at least 2).
    Beside it, the same oracle on one thread (the single-core figure the
    paper quotes its speed-ups against), for about a quarter of the budget
    (at least one step)."""
    import oracle
    case = workload(0)
    ncores = os.cpu_count() or 1

    def timed(nthreads, budget, min_steps):
        oracle.set_threads(nthreads)
        o = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                          case.eta_over_s, case.eos, nthreads=nthreads)
        o.set_initial(case.eps, case.ux, case.uy, case.ueta)
        steps = 0
        t0 = time.perf_counter()
        while steps < min_steps or (time.perf_counter() - t0 < budget and steps < 200):
            o.step(1)
            steps += 1
        return steps, time.perf_counter() - t0

    steps, dt = timed(ncores, budget_s, 2)
    out = {"value": case.ncells * steps / dt, "unit": UNIT, "cores": ncores, "kind": "oracle",
           "sample": f"{steps} full steps of the 97x97x41 event ({case.ncells} cells) in {dt:.1f} s, FP64, "
                     f"OpenMP over cells"}
    steps1, dt1 = timed(1, budget_s / 4, 1)
    out["single_thread"] = {"value": case.ncells * steps1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"{steps1} full steps of the same event in {dt1:.1f} s, FP64, one thread"}
    oracle.set_threads(ncores)
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    case = workload(0)
    ncores = os.cpu_count() or 1
    oracle.set_threads(ncores)
    o = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                      case.eta_over_s, case.eos, nthreads=ncores)
    o.set_initial(case.eps, case.ux, case.uy, case.ueta)
    steps = max(1, min(args.steps, 20))
    warm = max(0, min(args.warmup, 3))
    o.step(warm)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    v = case.ncells * steps / dt
    sample = f"{steps} full steps of the 97x97x41 event after {warm} warm-up steps, FP64, OpenMP over cells"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": steps,
        "warmup": warm, "ms_per_step": dt / steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "viscous hot-spot event 97x97x41, eta/s=0.08, crossover EOS table 4096, "
                               "2048 spots, b=7 fm, dtau=0.01 fm", "implementation": "FP64 CPU oracle"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": ncores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_slab(args):
    """--slab: one 261x261x121 mini-jet event split in x over the N ranks
    (x-slabs with halo exchange before every stage, NCCL point-to-point
    between neighbours; the stats are combined over the slabs in FP64).
    Strong scaling: the event is fixed, N GPUs share it.  FP32, previous-step
    guess; K timed steps after W warm-up steps, max over ranks."""
    import socket
    import torch
    import torch.distributed as dist
    from paper_1802_04449_gb300 import clv
    from paper_1802_04449_gb300 import inputs as I
    from paper_1802_04449_gb300 import slab as S

    ws, rank, local = dist_env()
    torch.cuda.set_device(local if ws > 1 else 0)
    if not dist.is_initialized():
        if ws == 1:   # a single-rank group: the same code path, no neighbour to exchange with
            sk = socket.socket()
            sk.bind(("127.0.0.1", 0))
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            os.environ.setdefault("MASTER_PORT", str(sk.getsockname()[1]))
            sk.close()
            dist.init_process_group("nccl", rank=0, world_size=1)
        else:
            dist.init_process_group("nccl")
    case = I.minijet_event()
    sl = S.DistSlab(case, rank, ws, clv.CLV_FP32)
    sl.step(args.warmup)
    torch.cuda.synchronize()
    dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = sl.h.stream
    e0.record(stream)
    sl.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    t = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = t.item()
    st = sl.step(1, stats=True)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": case.ncells * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "mode": "slab",
            "config": {"workload": "hot-spot event with mini-jet initial flow 261x261x121 split in x over the ranks",
                       "cells_per_event": case.ncells, "slab_planes": [n for _, n in S.partition(case.nx, ws)],
                       "parallelism": f"x-slabs over {ws} rank(s), halo exchange before every stage",
                       "guess": "previous-step"},
            "stats": {k: st.get(k) for k in ("tau", "eps_max", "T_max", "E_tot", "error_word")}}))
    dist.destroy_process_group()


def profile_case(args):
    """A short run through the C ABI for capture under a profiler: the
    kernels of interest are the last launches.  The event (--case: the
    97x97x41 hot-spot event, or the 261x261x121 mini-jet event) has its tile
    shape set by --tile or autotuned first (those timing launches come
    first), --skip steps
    run next (reaching a later, more dilute state), then --steps steps.
    --guess learned / learned-all trains the network briefly on FP64 states
    of another seed first.  --surface then takes a slice, runs 10 more steps,
    finds the freeze-out surface at T_f = 137 MeV between the two slices and
    computes the pi+, K+ and p spectra on the 41 x 15 x 48 grid from it: those
    launches come last.  --zeta-over-s Z > 0 evolves the bulk pressure too,
    --charge a smooth net charge."""
    import torch
    from paper_1802_04449_gb300 import clv
    from paper_1802_04449_gb300 import inputs as I
    from paper_1802_04449_gb300 import learned as L

    mk = I.minijet_event if args.case == "minijet" else I.hotspot_event
    case = mk()
    prec = clv.CLV_FP32 if args.precision == "fp32" else clv.CLV_FP64
    params = None
    if args.guess.startswith("learned"):
        tc = mk(seed=1000)
        h = clv.from_case(tc, clv.CLV_FP64)
        h.set_initial_case(tc)
        X, Y = L.collect_samples(h, max(args.skip + args.steps, 40), 20).data()
        p, _ = L.train(X, Y, iters=1000, batch=32768, lr=2e-3, seed=7)
        params = p.cpu().numpy()
        h.close()
        del X, Y
    g = clv.from_case(case, prec, zeta_over_s=args.zeta_over_s, charge=args.charge)
    g.set_initial_case(case)
    if args.charge:
        g.set_initial_n(0.2 + 0.05 * np.cos(np.linspace(0.0, 6.283, case.ncells)).reshape(case.eps.shape))
    if params is not None:
        g.set_mlp(params)
    g.set_guess({"previous": clv.CLV_GUESS_PREVIOUS, "cold": clv.CLV_GUESS_COLD, "learned": clv.CLV_GUESS_MLP,
                 "learned-all": clv.CLV_GUESS_MLP_ALL}[args.guess])
    if args.tile:
        g.set_tile(*(int(x) for x in args.tile.split(",")))
        print("tile:", g.tile())
    elif args.autotune:
        print("tile:", g.autotune(max_candidates=12, reps=3))
    if args.skip:
        g.step(args.skip)
    st = g.step(args.steps, stats=True)
    torch.cuda.synchronize()
    print("profile case done: tau %.3f, newton iters/solve %.3f, polished %d" %
          (st["tau"], st["n_newton_iters"] / max(1, st["n_newton_cells"]), st["n_polished"]))
    if args.surface:
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="clv", choices=["clv", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--batch-events", type=int, default=256,
                    help="events of the event-by-event batch measured beside the headline (0: skip)")
    ap.add_argument("--no-large", dest="large", action="store_false",
                    help="skip the 261x261x121 mini-jet event measured beside the headline")
    ap.add_argument("--no-lifetime", dest="lifetime", action="store_false",
                    help="skip the 261x261x121 event's run to max T < 137 MeV (FP32 + learned, then FP64)")
    ap.add_argument("--no-freezeout", dest="freezeout", action="store_false",
                    help="skip the freeze-out surface measured beside the headline")
    ap.add_argument("--no-options", dest="options", action="store_false",
                    help="skip the bulk-pressure and net-charge runs of the headline event")
    ap.add_argument("--no-accuracy", dest="accuracy", action="store_false",
                    help="skip the FP32-vs-FP64 accuracy check of the headline event")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default tile shape instead of timing candidates (setup, untimed)")
    ap.add_argument("--train-events", type=int, default=2, help="FP64 events whose states train the guess")
    ap.add_argument("--train-every", type=int, default=20, help="steps between sample dumps")
    ap.add_argument("--train-iters", type=int, default=4000, help="Adam iterations")
    pc = ap.add_argument_group("profile case (--profile-case: a short run for a profiler, no JSON line)")
    pc.add_argument("--profile-case", action="store_true")
    pc.add_argument("--case", default="hotspot", choices=["hotspot", "minijet"])
    pc.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    pc.add_argument("--guess", default="previous", choices=["previous", "cold", "learned", "learned-all"])
    pc.add_argument("--skip", type=int, default=0, help="steps before the profiled ones")
    pc.add_argument("--tile", default="", help="TJ,TK,CX of the stage kernel instead of autotuning")
    pc.add_argument("--surface", action="store_true")
    pc.add_argument("--zeta-over-s", type=float, default=0.0)
    pc.add_argument("--charge", action="store_true")
    ap.add_argument("--slab", action="store_true",
                    help="one 261x261x121 event split in x over the ranks (strong scaling) instead of the default")
    args = ap.parse_args()
    if args.slab:
        if args.warmup < 3:
            args.warmup = 3
        run_slab(args)
        return
    if args.profile_case:
        profile_case(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
