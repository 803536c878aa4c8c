"""Host side of the x-slab decomposition, on CPU: the partition and the
neighbour halo exchange over torch.distributed (gloo, three ranks)."""
import os
import socket

import numpy as np
import pytest

from paper_1802_04449_gb300 import slab as S


def test_partition():
    for nx in (4, 5, 97, 261):
        for parts in (1, 2, 3, 8):
            if nx < 2 * parts:
                with pytest.raises(ValueError):
                    S.partition(nx, parts)
                continue
            p = S.partition(nx, parts)
            assert [x for x, _ in p] == list(np.cumsum([0] + [n for _, n in p])[:-1])
            assert sum(n for _, n in p) == nx and min(n for _, n in p) >= 2
            assert max(n for _, n in p) - min(n for _, n in p) <= 1


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo = torch.full((5,), 10.0 * rank + 0.0)
        hi = torch.full((5,), 10.0 * rank + 1.0)
        rlo, rhi = S.exchange_halos(lo, hi, rank, world)
        st = S.reduce_stats(1.0 + rank * (rank - 1), 0.1 * rank, 10.0 ** rank)
        np.save(os.path.join(out, f"x{rank}.npy"),
                np.array([np.nan if rlo is None else float(rlo[0]), np.nan if rhi is None else float(rhi[0]),
                          st["eps_max"], st["T_max"], st["E_tot"]]))
    finally:
        dist.destroy_process_group()


def test_exchange_with_three_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 3
    mp.start_processes(_worker, args=(world, _port(), str(tmp_path)), nprocs=world, start_method="spawn")
    got = [np.load(tmp_path / f"x{r}.npy") for r in range(world)]
    # rank r receives the high planes of r - 1 and the low planes of r + 1
    assert np.isnan(got[0][0]) and got[0][1] == 10.0
    assert got[1][0] == 1.0 and got[1][1] == 20.0
    assert got[2][0] == 11.0 and np.isnan(got[2][1])
    # event statistics: the largest eps_max (rank 2: 3.0) with its T, E_tot summed
    for g in got:
        assert g[2] == 3.0 and g[3] == pytest.approx(0.2) and g[4] == 111.0


def test_combine_stats():
    got = S.combine_stats([(1.0, 0.2, 5.0), (4.0, 0.3, 6.0), (2.0, 0.25, 7.5)])
    assert got == {"eps_max": 4.0, "T_max": 0.3, "E_tot": 18.5}


def _leaving_worker(rank, world, port, out):
    """Rank 1 leaves between steps (exits before the next halo exchange);
    rank 0 must learn of it from the exchange itself, with an error instead
    of a hang (short process-group timeout)."""
    import datetime
    import sys

    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    lo = torch.full((5,), float(rank))
    hi = torch.full((5,), float(rank) + 0.5)
    S.exchange_halos(lo, hi, rank, world)          # one healthy exchange
    if rank == 1:
        sys.exit(0)                                # leaves with nothing in flight
    try:
        S.exchange_halos(lo, hi, rank, world)
        result = "no error"
    except Exception as e:                         # gloo reports the lost peer
        result = "detected: " + type(e).__name__
    with open(os.path.join(out, "rank0.txt"), "w") as f:
        f.write(result)


def test_a_rank_that_leaves_is_detected_by_its_neighbour(tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_leaving_worker, args=(2, _port(), str(tmp_path)), nprocs=2, start_method="spawn")
    assert (tmp_path / "rank0.txt").read_text().startswith("detected"), (tmp_path / "rank0.txt").read_text()


class _StandIn:
    """A CPU stand-in for an x-slab handle: one field with two halo planes on
    each x side and a stage that is a 5-point smoothing along x (different
    weights per stage), with the same slab calls as clv.Hydro."""

    def __init__(self, sub_case, precision=None, **kw):
        import torch
        self.device = torch.device("cpu")
        e = np.asarray(sub_case.eps, dtype=np.float64)
        self.n = e.shape[0]
        self.a = np.zeros((self.n + 4,) + e.shape[1:])
        self.a[2:self.n + 2] = e

    def halo_bytes(self):
        return 2 * self.a[0].size * 8

    def _planes(self, buf):
        return buf.numpy().view(np.float64).reshape((2,) + self.a.shape[1:])

    def slab_pack(self, set_, side, buf):
        self._planes(buf)[:] = self.a[2:4] if side == 0 else self.a[self.n:self.n + 2]

    def slab_unpack(self, set_, side, buf):
        if side == 0:
            self.a[0:2] = self._planes(buf)
        else:
            self.a[self.n + 2:] = self._planes(buf)

    def slab_fill_edge(self, set_, side):
        if side == 0:
            self.a[0:2] = self.a[2]
        else:
            self.a[self.n + 2:] = self.a[self.n + 1]

    def viscous_pending(self):
        return False

    def stage(self, s, stats=False):
        self.a[2:self.n + 2] = _smooth(self.a, s)
        if stats:
            x = self.a[2:self.n + 2]
            return {"eps_max": float(x.max()), "T_max": 0.0, "E_tot": float(x.sum())}
        return None


def _smooth(a, s):
    """The stand-in stage on a padded array: interior planes from their 5-point x neighbourhood."""
    w = (1.0, 2.0, 3.0, 2.0, 1.0) if s == 1 else (1.0, 1.0, 4.0, 1.0, 1.0)
    n = a.shape[0] - 4
    return sum(w[d] * a[d:d + n] for d in range(5)) / sum(w)


def _slab_loop_worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_1802_04449_gb300 import inputs as I
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = I.hotspot_event(nx=17, ny=4, neta=3, n_spots=6, seed=5)
        sl = S.DistSlab(case, rank, world, make=_StandIn)
        st = sl.step(6, stats=True)
        np.save(os.path.join(out, f"slab{rank}.npy"), sl.h.a[2:sl.h.n + 2])
        np.save(os.path.join(out, f"stats{rank}.npy"), np.array([st["eps_max"], st["E_tot"]]))
    finally:
        dist.destroy_process_group()


def test_stage_loop_through_the_exchange_with_three_gloo_ranks(tmp_path):
    """DistSlab's stage loop (pack, exchange with the x-neighbours, unpack or
    zero-gradient edge, stage) over three gloo ranks with a stand-in stage
    equals the same stages on the undivided grid, bit for bit, and the
    event statistics are combined over the slabs."""
    import torch.multiprocessing as mp
    from paper_1802_04449_gb300 import inputs as I
    world = 3
    mp.start_processes(_slab_loop_worker, args=(world, _port(), str(tmp_path)), nprocs=world, start_method="spawn")
    got = np.concatenate([np.load(tmp_path / f"slab{r}.npy") for r in range(world)], axis=0)
    case = I.hotspot_event(nx=17, ny=4, neta=3, n_spots=6, seed=5)
    a = np.zeros((case.nx + 4,) + case.eps.shape[1:])
    a[2:-2] = case.eps
    for _ in range(6):
        for s in (1, 2):
            a[0:2], a[-2:] = a[2], a[-3]
            a[2:-2] = _smooth(a, s)
    assert np.array_equal(got, a[2:-2])
    for r in range(world):
        st = np.load(tmp_path / f"stats{r}.npy")
        assert st[0] == a[2:-2].max() and st[1] == pytest.approx(a[2:-2].sum(), rel=1e-14)
