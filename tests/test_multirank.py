"""The N > 1 path on CPU ranks (gloo, world size 2): each rank evolves its
own events (sharded, seeds by global event index) with no data-path
collective; whole-job throughput = units summed over ranks / slowest rank.
Each rank runs the CPU oracle on a tiny event, so no GPU is needed."""
import os
import socket

import numpy as np
import pytest

from paper_1802_04449_gb300 import dist as D


def test_shard_covers_all_items_once():
    for n in (0, 1, 5, 256, 257):
        for w in (1, 2, 3, 8):
            got = [i for r in range(w) for i in D.shard(n, w, r)]
            assert got == list(range(n))
            sizes = [len(D.shard(n, w, r)) for r in range(w)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n_events, out_dir):
    import torch.distributed as dist
    import oracle
    from paper_1802_04449_gb300 import inputs as I
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        units = 0
        eps_sum = 0.0
        import time
        t0 = time.perf_counter()
        for ev in D.shard(n_events, world, rank):
            case = I.hotspot_event(nx=9, ny=9, neta=5, n_spots=12, seed=D.event_seed(100, ev))
            o = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                              case.eta_over_s, case.eos, nthreads=1)
            o.set_initial(case.eps, case.ux, case.uy, case.ueta)
            o.step(2)
            units += case.ncells * 2
            eps_sum += float(o.get("eps").sum())
        secs = time.perf_counter() - t0
        D.barrier()
        tp = D.throughput(units, secs)
        total_units = D.reduce_sum([units])[0]
        total_eps = D.reduce_sum([eps_sum])[0]
        np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([tp, total_units, total_eps, units, secs]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_events_and_aggregate(tmp_path):
    import torch.multiprocessing as mp
    world, n_events = 2, 5
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, n_events, str(tmp_path)), nprocs=world, start_method="spawn")
    r = [np.load(tmp_path / f"r{k}.npy") for k in range(world)]
    # both ranks agree on the aggregates
    assert r[0][0] == r[1][0] and r[0][1] == r[1][1] and r[0][2] == r[1][2]
    # the sharded run covers the same events as one rank doing them all
    import oracle
    from paper_1802_04449_gb300 import inputs as I
    ref_eps, ref_units = 0.0, 0
    for ev in range(n_events):
        case = I.hotspot_event(nx=9, ny=9, neta=5, n_spots=12, seed=D.event_seed(100, ev))
        o = oracle.Oracle(case.nx, case.ny, case.neta, case.dx, case.dy, case.deta, case.tau0, case.dtau,
                          case.eta_over_s, case.eos, nthreads=1)
        o.set_initial(case.eps, case.ux, case.uy, case.ueta)
        o.step(2)
        ref_eps += float(o.get("eps").sum())
        ref_units += case.ncells * 2
    assert r[0][1] == ref_units
    assert r[0][2] == pytest.approx(ref_eps, rel=1e-13)
    # throughput = total units / slowest rank
    assert r[0][0] == pytest.approx(ref_units / max(r[0][4], r[1][4]), rel=1e-12)
