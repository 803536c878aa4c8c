"""GPU path (libclv through its C ABI) against the FP64 oracle, element by
element on the same seeded inputs.

Tolerances:
  FP64 path: 1e-10 relative on every field, measured against the field's own
             magnitude (|g - o| <= 1e-10 (|o| + 1e-3 max|o|)), and 1e-10
             relative on eps wherever eps > 1e-3 GeV/fm^3.
  FP32 path: 1e-4 relative L-inf on eps wherever eps > 1e-3 GeV/fm^3.
"""
import numpy as np
import pytest

import oracle
from paper_1802_04449_gb300 import clv
from paper_1802_04449_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-4
EPS_FLOOR = 1e-3


def run_pair(case, nsteps, precision, pi=None, kernel=0):
    o = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                      case.eta_over_s, case.eos, case.cartesian, case.periodic)
    o.set_initial(case.eps, case.ux, case.uy, case.ueta, pi)
    o.step(nsteps)
    g = clv.from_case(case, precision, kernel=kernel)
    g.set_initial(case.eps, case.ux, case.uy, case.ueta, pi)
    st = g.step(nsteps, stats=True)
    return o, g, st


def compare_fp64(o, g, viscous, fields=None):
    names = fields or (["eps", "ux", "uy", "ueta", "Ttt", "Ttx", "Tty", "Tte"] +
                       ([k for k in clv.FIELDS if k.startswith("pi")] + ["upx", "upy", "upe"] if viscous else []))
    got = g.get(names)
    worst = {}
    for k in names:
        ref = o.get(k)
        scale = np.abs(ref).max()
        err = np.abs(got[k] - ref)
        bound = FP64_TOL * (np.abs(ref) + 1e-3 * scale) + 1e-300
        worst[k] = float((err / bound).max()) if scale > 0 else float(err.max())
        assert np.all(err <= bound) or (scale == 0 and err.max() == 0), (k, worst[k], err.max(), scale)
    e_o, e_g = o.get("eps"), got["eps"]
    m = e_o > EPS_FLOOR
    assert np.all(np.abs(e_g[m] / e_o[m] - 1) <= FP64_TOL)
    return worst


def fp32_eps_err(o, g):
    e_o = o.get("eps")
    e_g = g.get(["eps"])["eps"]
    m = e_o > EPS_FLOOR
    assert m.sum() > 0
    return float(np.max(np.abs(e_g[m] / e_o[m] - 1)))


# ------------------------------------------------------------------ cases
def small_hotspot(seed=3, nx=21, ny=19, neta=11, eta_over_s=0.08, nspots=60, eos="crossover"):
    return I.hotspot_event(nx=nx, ny=ny, neta=neta, n_spots=nspots, seed=seed, eta_over_s=eta_over_s,
                           eos=eos)


def test_fp64_gubser_ideal_config():
    """Ideal Gubser flow on the 33x33x9 grid, tau 1 -> 3 (100 steps)."""
    case = I.gubser_case()
    o, g, st = run_pair(case, case.nsteps, clv.CLV_FP64)
    compare_fp64(o, g, viscous=False)
    so = o.stats()
    assert st["tau"] == pytest.approx(so["tau"], rel=1e-14)
    assert st["eps_max"] == pytest.approx(so["eps_max"], rel=1e-10)
    assert st["E_tot"] == pytest.approx(so["E_tot"], rel=1e-10)
    assert st["error_word"] == 0


@pytest.mark.parametrize("eta_over_s,kernel", [(0.08, 0), (0.16, 0), (0.08, 1)])
def test_fp64_viscous_hotspots_table_eos(eta_over_s, kernel):
    case = small_hotspot(eta_over_s=eta_over_s)
    o, g, st = run_pair(case, 30, clv.CLV_FP64, kernel=kernel)
    compare_fp64(o, g, viscous=True)
    so = o.stats()
    assert st["E_tot"] == pytest.approx(so["E_tot"], rel=1e-10)
    assert st["T_max"] == pytest.approx(so["T_max"], rel=1e-10)


def test_fp64_viscous_longitudinal_flow_with_pi():
    """u~^eta != 0 (exercises I^{mu nu} and the eta flux) and a nonzero initial pi~."""
    rng = np.random.default_rng(9)
    nx, ny, ne = 9, 7, 24
    case = small_hotspot(nx=nx, ny=ny, neta=ne, nspots=20, eos=None, eta_over_s=0.16)
    eta = I.cell_coords(ne, case.deta)
    case.ueta = np.broadcast_to(0.2 * np.sin(eta), case.eps.shape).copy()
    case.ux = 0.05 * rng.normal(size=case.eps.shape)
    pi = 0.02 * rng.normal(size=(10,) + case.eps.shape) * case.eps   # small against the local eps
    o, g, st = run_pair(case, 25, clv.CLV_FP64, pi=pi)
    compare_fp64(o, g, viscous=True)


def test_fp64_shear_regulator_active():
    """Initial pi~ of the order of several eps, so that the shear regulator
    (|pi pi| <= eps^2 + 3P^2) acts in many cells during the first steps."""
    case = small_hotspot(seed=19, eta_over_s=0.16)
    pi = np.zeros((10,) + case.eps.shape)
    pi[4] = pi[7] = 2.0 * case.eps          # transverse, traceless for u = 0,
    pi[9] = -4.0 * case.eps                 # about 4x above the bound
    o, g, st = run_pair(case, 12, clv.CLV_FP64, pi=pi)
    compare_fp64(o, g, viscous=True)


def test_fp64_cartesian_periodic_box():
    rng = np.random.default_rng(4)
    e, ux, uy, ue = I.random_smooth_box(rng, 12, 10, 9)
    case = I.HydroCase("box", 12, 10, 9, 0.2, 0.2, 0.2, 1.0, 0.02, 0.16, None, e, ux, uy, ue, 40,
                       cartesian=True, periodic=True)
    o, g, st = run_pair(case, 40, clv.CLV_FP64)
    compare_fp64(o, g, viscous=True)
    keys = ["Ttt", "Ttx", "Tty", "Tte"]
    got = g.get(keys)
    ini = oracle.Oracle(12, 10, 9, 0.2, 0.2, 0.2, 1.0, 0.02, 0.16, cartesian=True, periodic=True)
    ini.set_initial(e, ux, uy, ue)
    for k in keys:   # GPU conserves sum T^{t mu} too
        assert abs(got[k].sum() - ini.get(k).sum()) <= 1e-12 * ini.get("Ttt").sum()


@pytest.mark.parametrize("shape", [(23, 29, 41), (16, 9, 70), (7, 40, 3)])
def test_tiled_kernel_matches_direct_kernel(shape):
    """The tiled kernel (several tiles, chunks and ragged edges) and the direct
    per-cell kernel run the same arithmetic: FP64 results agree to rounding."""
    nx, ny, ne = shape
    case = small_hotspot(nx=nx, ny=ny, neta=ne, nspots=80, seed=13)
    out = []
    for kern in (0, 1):
        g = clv.from_case(case, clv.CLV_FP64, kernel=kern)
        g.set_initial(case.eps, case.ux, case.uy, case.ueta)
        g.step(12)
        out.append(g.get())
    for k in out[0]:
        ref = out[1][k]
        scale = np.abs(ref).max()
        assert np.all(np.abs(out[0][k] - ref) <= 1e-12 * (np.abs(ref) + scale) + 1e-300), k


def test_fp64_riemann_vacuum_front():
    nx = 241
    x, e = I.riemann_1d(nx, 0.05, 10.0)
    sh = (nx, 1, 1)
    z = np.zeros(sh)
    case = I.HydroCase("riemann", nx, 1, 1, 0.05, 1.0, 1.0, 0.0, 0.0125, 0.0, None, e.reshape(sh), z, z, z,
                       200, cartesian=True)
    o, g, st = run_pair(case, 200, clv.CLV_FP64)
    compare_fp64(o, g, viscous=False)
    assert st["n_rescaled"] > 0   # the vacuum front exercises the |M| > E branch


@pytest.mark.parametrize("kernel", [0, 1])
def test_fp32_riemann_front_refinement(kernel):
    """The vacuum front drives cells to v -> 1 and to the cutoff: the FP32
    path refines them in FP64 (compacted second pass for the tiled path,
    inline for the direct kernel) and matches the oracle within 1e-4 where
    eps > 1e-3 GeV/fm^3."""
    nx = 241
    x, e = I.riemann_1d(nx, 0.05, 10.0)
    sh = (nx, 1, 1)
    z = np.zeros(sh)
    case = I.HydroCase("riemann", nx, 1, 1, 0.05, 1.0, 1.0, 0.0, 0.0125, 0.0, None, e.reshape(sh), z, z, z,
                       200, cartesian=True)
    o, g, st = run_pair(case, 200, clv.CLV_FP32, kernel=kernel)
    assert st["n_polished"] > 0 and st["n_rootfail"] == 0 and st["error_word"] == 0
    assert fp32_eps_err(o, g) <= FP32_TOL
    # the velocity at the front: u~^x relative error where eps > 1e-3
    e_o = o.get("eps")
    m = e_o > EPS_FLOOR
    u_o, u_g = o.get("ux")[m], g.get(["ux"])["ux"][m]
    assert np.max(np.abs(u_g - u_o) / (np.abs(u_o) + 1e-3)) <= 1e-3


@pytest.mark.parametrize("eos,kernel", [("crossover", 0), (None, 0), ("crossover", 1)])
def test_fp32_viscous_hotspots(eos, kernel):
    case = small_hotspot(seed=7, eos=eos)
    o, g, st = run_pair(case, 40, clv.CLV_FP32, kernel=kernel)
    err = fp32_eps_err(o, g)
    assert err <= FP32_TOL, err
    assert st["error_word"] == 0


def test_fp32_gubser():
    case = I.gubser_case()
    o, g, st = run_pair(case, case.nsteps, clv.CLV_FP32)
    assert fp32_eps_err(o, g) <= FP32_TOL


def test_full_size_viscous_event_one_step():
    """The 97x97x41 viscous hot-spot event (2048 spots, crossover EOS) in the
    launch configuration the benchmark times: one full step, every cell."""
    case = I.hotspot_event()
    oracle.set_threads(0)
    o, g64, _ = run_pair(case, 1, clv.CLV_FP64)
    compare_fp64(o, g64, viscous=True, fields=["eps", "ux", "uy", "ueta", "Ttt", "Tte", "pixx", "piee"])
    g32 = clv.from_case(case, clv.CLV_FP32)
    g32.set_initial(case.eps, case.ux, case.uy, case.ueta)
    g32.step(1)
    assert fp32_eps_err(o, g32) <= FP32_TOL


LARGEST_STEPS = 24


def test_largest_event_24_steps():
    """The largest configuration, the 261x261x121 mini-jet event (8.2 M cells,
    initial state from T^{tau mu}, eta/s = 0.16): 24 full steps (about a
    minute of oracle time on the host's cores), every cell, FP64 to the FP64
    bar and FP32 (the benchmark's precision) to the FP32 bar."""
    case = I.minijet_event()
    oracle.set_threads(0)
    o = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                      case.eta_over_s, case.eos, case.cartesian, case.periodic)
    o.set_initial_T(case.T0)
    o.step(LARGEST_STEPS)
    g64 = clv.from_case(case, clv.CLV_FP64)
    g64.set_initial_case(case)
    st = g64.step(LARGEST_STEPS, stats=True)
    assert st["error_word"] == 0
    compare_fp64(o, g64, viscous=True, fields=["eps", "ux", "ueta", "Ttt", "Ttx", "pixx", "piee"])
    g64.close()
    g32 = clv.from_case(case, clv.CLV_FP32)
    g32.set_initial_case(case)
    st = g32.step(LARGEST_STEPS, stats=True)
    assert st["error_word"] == 0
    assert fp32_eps_err(o, g32) <= FP32_TOL
    g32.close()


def test_single_cell_and_degenerate_grids():
    for shape in [(1, 1, 1), (1, 1, 5), (3, 1, 1), (2, 3, 1)]:
        nx, ny, ne = shape
        e = np.full(shape, 4.0)
        e.flat[0] = 6.0
        z = np.zeros(shape)
        case = I.HydroCase("tiny", nx, ny, ne, 0.3, 0.3, 0.3, 0.6, 0.02, 0.1, None, e, z, z, z, 5)
        o, g, st = run_pair(case, 5, clv.CLV_FP64)
        compare_fp64(o, g, viscous=True)


def test_device_inputs_equal_host_inputs_and_deterministic():
    import torch
    case = small_hotspot(seed=11)
    g1 = clv.from_case(case, clv.CLV_FP32)
    g1.set_initial(case.eps, case.ux, case.uy, case.ueta)
    g1.step(10)
    a = g1.get()
    g2 = clv.from_case(case, clv.CLV_FP32, torch_workspace=False)
    dev = [torch.tensor(x, device="cuda") for x in (case.eps, case.ux, case.uy, case.ueta)]
    g2.set_initial(*dev)
    g2.step(10)
    b = g2.get()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_error_paths():
    with pytest.raises(clv.ClvError) as ei:
        clv.Hydro(0, 4, 4, 0.1, 0.1, 0.1, 1.0, 0.01)
    assert ei.value.status == 1
    with pytest.raises(clv.ClvError):
        clv.Hydro(4, 4, 4, 0.1, 0.1, 0.1, -1.0, 0.01)   # tau0 <= 0 in Milne coordinates
    g = clv.Hydro(4, 4, 4, 0.1, 0.1, 0.1, 1.0, 0.01)
    with pytest.raises(clv.ClvError):
        g.step(1)                                        # no initial state yet
    e = np.full((4, 4, 4), 5.0)
    z = np.zeros_like(e)
    ux = z.copy()
    ux[1, 2, 3] = np.nan                                 # non-finite input is reported
    g.set_initial(e, ux, z, z)
    with pytest.raises(clv.ClvError) as ei:
        g.step(2, stats=True)
    assert ei.value.status == 5


def test_device_arguments_are_checked():
    """CUDA tensors of the wrong size, or in host memory, are refused before
    the C call (CLV_EINVAL); tensors of the right size still work."""
    import torch
    g = clv.Hydro(4, 4, 4, 0.1, 0.1, 0.1, 1.0, 0.01, eta_over_s=0.1)
    ok = torch.full((4, 4, 4), 5.0, dtype=torch.float64, device=g.device)
    z = torch.zeros_like(ok)
    for bad in ((ok[:3], z, z, z), (ok, z, z, z.flatten()[:63])):
        with pytest.raises(clv.ClvError) as ei:
            g.set_initial(*bad)
        assert ei.value.status == 1
    with pytest.raises(clv.ClvError):
        g.set_initial(ok, z, z, z, torch.zeros(9 * 64, dtype=torch.float64, device=g.device))   # pi: 10 x 64
    with pytest.raises(clv.ClvError):
        g.set_initial_T(torch.zeros(3 * 64, dtype=torch.float64, device=g.device))
    g.set_initial(ok, z, z, z, torch.zeros(10 * 64, dtype=torch.float64, device=g.device))
    assert g.step(1, stats=True)["error_word"] == 0
    with pytest.raises(clv.ClvError):
        g.mlp_forward(torch.zeros((5, 9), device=g.device))
    with pytest.raises(clv.ClvError):
        g.mlp_forward(torch.zeros((5, 10)))                  # host memory


def test_tile_shapes_and_autotuner_leave_results_unchanged():
    """The tile shape is a schedule, not arithmetic: explicit shapes and the
    autotuner's choice give bit-identical fields to the default shape."""
    case = small_hotspot(seed=9, nx=23, ny=21, neta=13)
    names = ["eps", "ux", "uy", "ueta", "pixx", "piee"]

    def run(prec, shape=None, tune=False):
        g = clv.from_case(case, prec)
        g.set_initial(case.eps, case.ux, case.uy, case.ueta)
        if shape is not None:
            g.set_tile(*shape)
        if tune:
            info = g.autotune(max_candidates=6, reps=2)
            assert info["ms"] > 0 and info["threads"] == (info["TJ"] + 1) * (info["TK"] + 1)
        g.step(4)
        return g.get(names), g.tile()

    for prec in (clv.CLV_FP64, clv.CLV_FP32):
        ref, t0 = run(prec)
        for shape in ((3, 5, 0), (1, 13, 4), (7, 2, 23), (21, 1, 1)):
            got, t = run(prec, shape)
            assert (t["TJ"], t["TK"]) == shape[:2]
            for k in names:
                assert np.array_equal(got[k], ref[k]), (prec, shape, k)
        got, t = run(prec, tune=True)
        for k in names:
            assert np.array_equal(got[k], ref[k]), (prec, "autotuned", t, k)
    g = clv.from_case(case, clv.CLV_FP32)
    g.set_initial(case.eps, case.ux, case.uy, case.ueta)
    for bad in ((0, 5, 0), (3, 14, 0), (3, 5, 24)):
        with pytest.raises(clv.ClvError):
            g.set_tile(*bad)
    # more threads per CTA than the stage kernel is built for (384 in FP32)
    wide = small_hotspot(seed=9, nx=9, ny=40, neta=13)
    g = clv.from_case(wide, clv.CLV_FP32)
    g.set_initial(wide.eps, wide.ux, wide.uy, wide.ueta)
    with pytest.raises(clv.ClvError):
        g.set_tile(30, 13, 0)
    g.set_tile(20, 13, 0)   # 21 x 14 = 294 threads: allowed


@pytest.mark.parametrize("eta_over_s,prec", [(0.0, clv.CLV_FP64), (0.16, clv.CLV_FP64), (0.16, clv.CLV_FP32)])
def test_minijet_initial_flow(eta_over_s, prec):
    """Initial state from T^{tau mu} with transverse momentum (mini-jet
    flow): the GPU's root solve of the initial state and the evolution
    against the oracle's."""
    case = I.minijet_event(nx=19, ny=17, neta=9, dx=0.2, deta=0.2, n_spots=40, seed=12, eta_over_s=eta_over_s,
                           dtau=0.01)
    o = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                      case.eta_over_s, case.eos)
    o.set_initial_T(case.T0)
    g = clv.from_case(case, prec)
    g.set_initial_T(case.T0)
    if prec == clv.CLV_FP64:
        compare_fp64(o, g, viscous=eta_over_s > 0)      # the initial state itself
    o.step(6)
    st = g.step(6, stats=True)
    assert st["error_word"] == 0
    if prec == clv.CLV_FP64:
        compare_fp64(o, g, viscous=eta_over_s > 0)
    else:
        assert fp32_eps_err(o, g) <= FP32_TOL
    # device input equals host input
    import torch
    g2 = clv.from_case(case, prec)
    g2.set_initial_T(torch.tensor(case.T0, device="cuda"))
    g2.step(6)
    assert np.array_equal(g2.get(["eps"])["eps"], g.get(["eps"])["eps"])


def test_minijet_initial_state_errors():
    case = I.minijet_event(nx=9, ny=9, neta=5, dx=0.2, deta=0.2, n_spots=10, seed=2)
    g = clv.from_case(case, clv.CLV_FP64)
    bad = case.T0.copy()
    bad[1, 4, 4, 2] = np.nan
    with pytest.raises(clv.ClvError) as e:
        g.set_initial_T(bad)
    assert e.value.status == 5          # CLV_ENONFINITE
    g.set_initial_T(case.T0)          # the handle stays usable
    assert g.step(1, stats=True)["error_word"] == 0


@pytest.mark.parametrize("prec", [clv.CLV_FP64, clv.CLV_FP32])
def test_checkpoint_restart_is_bitwise(prec):
    """get_state after 7 steps, restore into a fresh handle: 5 more steps
    there equal 5 more steps of the original run bit for bit."""
    case = small_hotspot(seed=17)
    a = clv.from_case(case, prec)
    a.set_initial(case.eps, case.ux, case.uy, case.ueta)
    a.step(7)
    state = a.get_state()
    a.step(5)
    b = clv.from_case(case, prec)
    b.set_state(state)
    assert b.time()[0] == pytest.approx(case.tau0 + 7 * case.dtau, rel=1e-14) and b.time()[1] == 7
    b.step(5)
    names = ["eps", "ux", "uy", "ueta", "Ttt", "Tte", "pixx", "pixe", "upx"]
    ra, rb = a.get(names), b.get(names)
    for k in names:
        assert np.array_equal(ra[k], rb[k]), k
    assert a.time() == b.time()
    # another configuration is refused
    other = small_hotspot(seed=17, nx=19)
    c = clv.from_case(other, prec)
    with pytest.raises(clv.ClvError):
        c.set_state(state)
    with pytest.raises(clv.ClvError):
        b.set_state(state[:100])


@pytest.mark.parametrize("prec", [clv.CLV_FP64, clv.CLV_FP32])
def test_batch_of_uneven_events_equals_single_events(prec):
    """Events of different grids and eta/s (ideal and viscous) in one batch:
    one persistent stage launch and one root-solve launch per stage give
    each event the fields of its own single-event run -- the same stage body
    and root solve, so FP64 agrees bit for bit and FP32 to its rounding (the
    batched kernel is a separate instantiation, free to contract products
    into fused multiply-adds differently)."""
    cases = [
        I.hotspot_event(nx=23, ny=21, neta=13, n_spots=60, seed=41, eta_over_s=0.08),
        I.hotspot_event(nx=17, ny=25, neta=7, dx=0.25, deta=0.25, n_spots=40, seed=42, eta_over_s=0.0),
        I.hotspot_event(nx=31, ny=19, neta=41, dx=0.15, deta=0.15, n_spots=80, seed=43, eta_over_s=0.16),
        I.hotspot_event(nx=5, ny=3, neta=1, n_spots=4, seed=44, eta_over_s=0.08),
    ]
    nsteps = 5
    b = clv.Batch(cases, prec)
    assert b.nevents == 4 and b.N == sum(c.ncells for c in cases)
    for e, c in enumerate(cases):
        b.set_event(e, c.eps, c.ux, c.uy, c.ueta)
    b.step(1)
    b.enable_kernel_timing(True)       # per-kernel events: four slots per step, all filled
    st = b.step(nsteps - 1, stats=True)
    kt = b.kernel_times()
    assert all(n == nsteps - 1 and ms > 0 for ms, n in kt.values()), kt
    assert st["error_word"] == 0 and st["E_tot"] == 0.0
    names = ["eps", "ux", "uy", "ueta", "Ttt", "Ttx", "Tte", "pixx", "pixy", "piee", "upx"]
    for e, c in enumerate(cases):
        g = clv.from_case(c, prec)
        g.set_initial(c.eps, c.ux, c.uy, c.ueta)
        sg = g.step(nsteps, stats=True)
        ref, got = g.get(names), b.get_event(e, names)
        # FP32: the batched kernel rounds differently (its own register
        # allocation and contractions), by about one unit in the last place of
        # each operation; after a few steps that is ~1e-6 of a field's scale
        rtol, floor = (0.0, 1e-3) if prec == clv.CLV_FP64 else (2e-6, 1.0)
        for k in names:
            scale = np.abs(ref[k]).max()
            dev = float((np.abs(got[k] - ref[k]) / (np.abs(ref[k]) + floor * scale + 1e-300)).max())
            assert dev <= rtol, (e, k, dev)
        es = b.event_stats(e)
        assert es["eps_max"] == pytest.approx(sg["eps_max"], rel=rtol)
        assert es["E_tot"] == pytest.approx(sg["E_tot"], rel=max(rtol, 1e-12))
    # calls that do not apply to a batch
    flat = np.zeros(b.N)
    with pytest.raises(clv.ClvError):
        b.set_initial(flat, flat, flat, flat)
    with pytest.raises(clv.ClvError):
        b.set_tile(4, 4, 4)
    with pytest.raises(clv.ClvError):
        b.set_event(0, cases[0].eps, cases[0].ux, cases[0].uy, cases[0].ueta)   # already started


@pytest.mark.parametrize("prec", [clv.CLV_FP64, clv.CLV_FP32])
def test_batch_schedules_and_autotuner_leave_results_unchanged(prec):
    """Tiling policies of a batch (thread cap, x chunk), explicit or picked by
    the autotuner between steps, give bit-identical fields."""
    cases = [
        I.hotspot_event(nx=23, ny=21, neta=13, n_spots=60, seed=41, eta_over_s=0.08),
        I.hotspot_event(nx=17, ny=25, neta=7, dx=0.25, deta=0.25, n_spots=40, seed=42, eta_over_s=0.0),
        I.hotspot_event(nx=31, ny=19, neta=41, dx=0.15, deta=0.15, n_spots=80, seed=43, eta_over_s=0.16),
    ]
    names = ["eps", "ux", "ueta", "Ttt", "pixx", "piee"]
    runs = []
    for sched in (None, (128, 8), (64, 48), "tune"):
        b = clv.Batch(cases, prec)
        for e, c in enumerate(cases):
            b.set_event(e, c.eps, c.ux, c.uy, c.ueta)
        if sched == "tune":
            with pytest.raises(clv.ClvError):
                b.autotune()                     # the batch starts at its first step
        elif sched is not None:
            b.set_schedule(*sched)
        b.step(3)
        if sched == "tune":
            info = b.autotune(max_candidates=8, reps=2)
            assert info["TK"] == 0 and info["TJ"] >= 32 and info["CX"] >= 1 and info["ms"] > 0
            assert b.tile() == {**info, "ms": 0.0}
        b.step(3)
        runs.append([b.get_event(e, names) for e in range(len(cases))])
        b.close()
    for r in runs[1:]:
        for e in range(len(cases)):
            for k in names:
                np.testing.assert_array_equal(r[e][k], runs[0][e][k])
    b = clv.Batch(cases[:1], prec)
    with pytest.raises(clv.ClvError):
        b.set_schedule(16, 32)                   # thread cap below a warp
    with pytest.raises(clv.ClvError):
        b.set_schedule(256, 0)
    b.close()


def test_batch_needs_every_event_and_a_common_setup():
    a = I.hotspot_event(nx=9, ny=9, neta=5, n_spots=10, seed=1)
    c = I.hotspot_event(nx=11, ny=7, neta=3, n_spots=10, seed=2)
    b = clv.Batch([a, c], clv.CLV_FP64)
    b.set_event(0, a.eps, a.ux, a.uy, a.ueta)
    with pytest.raises(clv.ClvError):
        b.step(1)                                  # event 1 has no initial state
    d = I.hotspot_event(nx=9, ny=9, neta=5, n_spots=10, seed=3, dtau=0.02)
    with pytest.raises(clv.ClvError):
        clv.Batch([a, d], clv.CLV_FP64)            # different dtau


@pytest.mark.parametrize("prec,eta_over_s", [(clv.CLV_FP64, 0.08), (clv.CLV_FP32, 0.16), (clv.CLV_FP32, 0.0)])
def test_step_graphs_equal_direct_launches(prec, eta_over_s):
    """Pairs of steps replayed from a captured graph (tau on the device) give
    the fields and tau of directly launched steps bit for bit, with stats
    steps and odd counts interleaved, and on a non-default stream."""
    import torch
    case = small_hotspot(seed=23, eta_over_s=eta_over_s)
    runs = []
    for graphs, stream in ((False, None), (True, None), (True, torch.cuda.Stream())):
        g = clv.from_case(case, prec, stream=stream)
        g.set_graphs(graphs)
        g.set_initial(case.eps, case.ux, case.uy, case.ueta)
        g.step(5)
        st = g.step(4, stats=True)
        g.step(3)
        runs.append((g.get(["eps", "ux", "ueta", "Ttt", "pixy"]), g.time(), st))
    for fields, t, st in runs[1:]:
        assert t == runs[0][1]
        assert st["eps_max"] == runs[0][2]["eps_max"] and st["E_tot"] == runs[0][2]["E_tot"]
        for k in fields:
            assert np.array_equal(fields[k], runs[0][0][k]), k


@pytest.mark.parametrize("prec", [clv.CLV_FP64, clv.CLV_FP32])
def test_viscous_gubser_lambda1(prec):
    """Second-order viscous Gubser flow (lambda_1 term, tau_pi from the
    solution's constraint) on the GPU against the oracle, and the GPU run
    against the analytic solution in the core."""
    case = I.gubser_viscous_case(dx=0.2, nx=41, neta=3, deta=0.2, dtau=0.01, tau1=1.5)
    o = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                      case.eta_over_s, None, taupi_coef=case.taupi_coef, lambda1_hat=case.lambda1_hat)
    o.set_initial(case.eps, case.ux, case.uy, case.ueta, case.pi0)
    o.step(case.nsteps)
    g = clv.from_case(case, prec)
    g.set_initial_case(case)
    st = g.step(case.nsteps, stats=True)
    assert st["error_word"] == 0
    if prec == clv.CLV_FP64:
        compare_fp64(o, g, viscous=True)
    else:
        assert fp32_eps_err(o, g) <= FP32_TOL
    x = I.cell_coords(case.nx, case.dx)
    e, ux, uy, pi = I.gubser_viscous(1.5, x, x)
    X, Y = np.meshgrid(x, x, indexing="ij")
    core = np.sqrt(X * X + Y * Y) <= 2.0
    got = g.get(["eps", "pixx"])
    assert np.abs(got["eps"][:, :, 1][core] / e[core] - 1).mean() < 2e-2
    assert np.abs(got["pixx"][:, :, 1][core] - pi[4][core]).mean() < 2e-2 * np.abs(pi[4][core]).mean()


@pytest.mark.parametrize("prec,eta_over_s,parts", [(clv.CLV_FP64, 0.08, 2), (clv.CLV_FP64, 0.16, 3),
                                                   (clv.CLV_FP32, 0.08, 2), (clv.CLV_FP64, 0.0, 3)])
def test_x_slabs_equal_the_single_domain(prec, eta_over_s, parts):
    """An event split into x-slabs (halo planes exchanged before every stage,
    zero-gradient copies at the global ends) evolves exactly as the single
    domain: every field bit for bit, the first-step predictor included."""
    from paper_1802_04449_gb300 import slab as S
    case = small_hotspot(seed=29, nx=25, ny=19, neta=11, eta_over_s=eta_over_s)
    g = clv.from_case(case, prec)
    g.set_initial(case.eps, case.ux, case.uy, case.ueta)
    g.step(6)
    sl = S.LocalSlabs(case, parts, prec)
    sl.step(6)
    names = ["eps", "ux", "uy", "ueta", "Ttt", "Ttx", "Tte"] + (["pixx", "pixe", "piee", "upx", "upe"]
                                                               if eta_over_s > 0 else [])
    ref, got = g.get(names), sl.get(names)
    for k in names:
        assert np.array_equal(got[k], ref[k]), k
    assert sl.slabs[0].time() == g.time()
    with pytest.raises(clv.ClvError):
        sl.slabs[0].step(1)                      # an x-slab steps by stages


def test_x_slab_mini_jet_initial_state():
    """The T^{tau mu} initial state of a slab (its own root solves) and its
    evolution equal the single domain's."""
    from paper_1802_04449_gb300 import slab as S
    case = I.minijet_event(nx=20, ny=15, neta=7, dx=0.2, deta=0.2, n_spots=30, seed=5, eta_over_s=0.16,
                           dtau=0.01)
    g = clv.from_case(case, clv.CLV_FP64)
    g.set_initial_T(case.T0)
    g.step(4)
    sl = S.LocalSlabs(case, 2, clv.CLV_FP64)
    sl.step(4)
    for k in ("eps", "ux", "pixy"):
        assert np.array_equal(sl.get([k])[k], g.get([k])[k]), k


def test_dist_slab_on_one_rank_equals_the_single_domain():
    """The path bench.py --slab times: DistSlab on a one-rank NCCL group (no
    neighbour, zero-gradient edges, the stats combined by all_gather) gives
    the single domain's fields bit for bit, FP32 and FP64."""
    import os
    import socket

    import torch
    import torch.distributed as dist
    from paper_1802_04449_gb300 import slab as S
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(sk.getsockname()[1])
    sk.close()
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        case = small_hotspot(seed=12, nx=15, ny=13, neta=9, eta_over_s=0.08)
        for prec in (clv.CLV_FP64, clv.CLV_FP32):
            sl = S.DistSlab(case, 0, 1, prec)
            st = sl.step(5, stats=True)
            g = clv.from_case(case, prec)
            g.set_initial(case.eps, case.ux, case.uy, case.ueta)
            sg = g.step(5, stats=True)
            for k in ("eps", "ux", "ueta", "pixx", "piee"):
                assert np.array_equal(sl.h.get([k])[k], g.get([k])[k]), (prec, k)
            assert st["eps_max"] == sg["eps_max"] and st["E_tot"] == pytest.approx(sg["E_tot"], rel=1e-12)
    finally:
        dist.destroy_process_group()


def test_fma_rate_is_a_plausible_peak():
    """clv_fma_rate (the ALU-roofline denominator) measures the FMA rate of
    this GPU: FP32 far above FP64, both within a factor of two of the
    GB300's nominal rates (FP32 152 SMs x 128 lanes x 2 x ~2 GHz = 80
    TFLOP/s, FP64 1.25 TFLOP/s); other precisions are refused."""
    f64 = clv.fma_rate(clv.CLV_FP64)
    f32 = clv.fma_rate(clv.CLV_FP32)
    assert 0.6 < f64 < 2.5, f64
    assert 40.0 < f32 < 160.0, f32
    with pytest.raises(clv.ClvError):
        clv.fma_rate(7)
