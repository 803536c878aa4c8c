"""One event split into slabs along x, one per GPU (the outermost axis of the
layout): partition, halo exchange and the stage loop around the C ABI's
x-slab calls (clv_slab_*, clv_stage).

Every stage reads two planes beyond each x end of its slab.  Before stage s
each slab packs the two boundary planes of the fields stage s reads (set s),
sends them to its neighbours and unpacks theirs into its halo planes; the
ends of the global grid get zero-gradient copies instead (clv_slab_fill_edge).
DistSlab exchanges with torch.distributed point-to-point messages (NCCL on
GPUs, gloo on CPU); LocalSlabs keeps all slabs of an event on one device and
exchanges by device copies."""
from __future__ import annotations

from dataclasses import replace

import numpy as np

from . import clv


def partition(nx, parts):
    """Balanced split of nx planes into `parts` slabs: [(x_begin, nx_local)],
    every slab at least 2 planes wide."""
    if parts < 1 or nx < 2 * parts:
        raise ValueError("need at least two x planes per slab")
    base, extra = divmod(nx, parts)
    out, x = [], 0
    for r in range(parts):
        n = base + (1 if r < extra else 0)
        out.append((x, n))
        x += n
    return out


def slab_case(case, x_begin, nloc):
    """The sub-event of planes [x_begin, x_begin + nloc) (initial fields sliced)."""
    sl = slice(x_begin, x_begin + nloc)
    kw = dict(nx=nloc, eps=case.eps[sl], ux=case.ux[sl], uy=case.uy[sl], ueta=case.ueta[sl])
    if getattr(case, "pi0", None) is not None:
        kw["pi0"] = case.pi0[:, sl]
    if getattr(case, "T0", None) is not None:
        kw["T0"] = case.T0[:, sl]
    return replace(case, **kw)


def exchange_halos(send_lo, send_hi, rank, world, group=None):
    """Swap boundary planes with the x-neighbours: send_lo goes to rank - 1,
    send_hi to rank + 1; returns (recv_lo, recv_hi) from rank - 1 and rank + 1
    (None at the ends of the global grid)."""
    import torch
    import torch.distributed as dist
    ops, recv_lo, recv_hi = [], None, None
    if rank > 0:
        recv_lo = torch.empty_like(send_lo)
        ops.append(dist.P2POp(dist.isend, send_lo, rank - 1, group))
        ops.append(dist.P2POp(dist.irecv, recv_lo, rank - 1, group))
    if rank < world - 1:
        recv_hi = torch.empty_like(send_hi)
        ops.append(dist.P2POp(dist.isend, send_hi, rank + 1, group))
        ops.append(dist.P2POp(dist.irecv, recv_hi, rank + 1, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    return recv_lo, recv_hi


def combine_stats(parts):
    """Event statistics from per-slab (eps_max, T_max, E_tot): the largest
    eps_max with its temperature, and the FP64 sum of E_tot."""
    e, t, _ = max(parts, key=lambda p: p[0])
    return {"eps_max": e, "T_max": t, "E_tot": float(np.sum([p[2] for p in parts], dtype=np.float64))}


def reduce_stats(eps_max, T_max, E_tot, device=None, group=None):
    """combine_stats over all ranks (all_gather of three FP64 values)."""
    import torch
    import torch.distributed as dist
    mine = torch.tensor([eps_max, T_max, E_tot], dtype=torch.float64, device=device)
    got = [torch.empty_like(mine) for _ in range(dist.get_world_size(group))]
    dist.all_gather(got, mine, group=group)
    return combine_stats([tuple(g.tolist()) for g in got])


def _new_slab(case, precision, **kw):
    h = clv.from_case(case, precision, halo_x=2, **kw)
    h.set_initial_case(case)
    return h


class DistSlab:
    """This rank's slab of an event (torch.distributed initialised, one rank
    per slab, slabs in rank order along x).  ``make(sub_case, precision,
    **kw)`` builds the slab's handle (an x-slab clv.Hydro by default; any
    object with the same slab calls works, which lets the stage loop and the
    exchange be tested on CPU)."""

    def __init__(self, case, rank, world, precision=clv.CLV_FP64, group=None, make=None, **kw):
        import torch
        self.rank, self.world, self.group = rank, world, group
        self.x_begin, self.nx = partition(case.nx, world)[rank]
        self.h = (make or _new_slab)(slab_case(case, self.x_begin, self.nx), precision, **kw)
        n = self.h.halo_bytes()
        self._send = [torch.empty(n, dtype=torch.uint8, device=self.h.device) for _ in range(2)]
        if self.h.viscous_pending():
            for s in (1, 2):
                self._halos(s)
                self.h.slab_predictor(s)

    def _halos(self, set_):
        self.h.slab_pack(set_, 0, self._send[0])
        self.h.slab_pack(set_, 1, self._send[1])
        lo, hi = exchange_halos(self._send[0], self._send[1], self.rank, self.world, self.group)
        for side, buf in ((0, lo), (1, hi)):
            if buf is None:
                self.h.slab_fill_edge(set_, side)
            else:
                self.h.slab_unpack(set_, side, buf)

    def step(self, n=1, stats=False):
        """n steps; with stats, the event's eps_max, T_max and E_tot over all
        slabs after the last step (and this slab's counters)."""
        st = None
        for k in range(n):
            for s in (1, 2):
                self._halos(s)
                st = self.h.stage(s, stats=stats and s == 2 and k == n - 1)
        if st is not None:
            st.update(reduce_stats(st["eps_max"], st["T_max"], st["E_tot"], self.h.device, self.group))
        return st


class LocalSlabs:
    """All slabs of an event on one device, exchanging halos by copies."""

    def __init__(self, case, parts, precision=clv.CLV_FP64, **kw):
        import torch
        self.parts = partition(case.nx, parts)
        self.slabs = [_new_slab(slab_case(case, x0, n), precision, **kw) for x0, n in self.parts]
        nb = self.slabs[0].halo_bytes()
        self._buf = [[torch.empty(nb, dtype=torch.uint8, device=self.slabs[0].device) for _ in range(2)]
                     for _ in self.slabs]
        if self.slabs[0].viscous_pending():
            for s in (1, 2):
                self._halos(s)
                for h in self.slabs:
                    h.slab_predictor(s)

    def _halos(self, set_):
        for h, (lo, hi) in zip(self.slabs, self._buf):
            h.slab_pack(set_, 0, lo)
            h.slab_pack(set_, 1, hi)
        last = len(self.slabs) - 1
        for k, h in enumerate(self.slabs):
            if k == 0:
                h.slab_fill_edge(set_, 0)
            else:
                h.slab_unpack(set_, 0, self._buf[k - 1][1])
            if k == last:
                h.slab_fill_edge(set_, 1)
            else:
                h.slab_unpack(set_, 1, self._buf[k + 1][0])

    def step(self, n=1):
        for _ in range(n):
            for s in (1, 2):
                self._halos(s)
                for h in self.slabs:
                    h.stage(s)

    def get(self, names):
        parts = [h.get(names) for h in self.slabs]
        return {k: np.concatenate([p[k] for p in parts], axis=0) for k in parts[0]}
