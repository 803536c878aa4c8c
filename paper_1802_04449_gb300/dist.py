"""Multi-rank helpers: events are independent problems, so they are sharded
across ranks with no data-path collective.  The only collectives are the
timing barrier and the reductions of the timing and the unit counts.

One process per GPU, launched by torchrun; RANK / WORLD_SIZE / LOCAL_RANK
come from the environment.
"""
from __future__ import annotations

import os


def env():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_items: int, world: int, rank: int) -> range:
    """Contiguous, balanced block of item indices owned by ``rank``."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    base, extra = divmod(n_items, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def event_seed(base: int, index: int) -> int:
    """Seed of global event ``index`` (the same event on any rank count)."""
    return base + index


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def barrier():
    d = _dist()
    if d is not None:
        d.barrier()


def reduce_max(values, device=None):
    """Element-wise max over ranks of a list of floats (identity on one rank)."""
    import torch
    d = _dist()
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if d is not None:
        d.all_reduce(t, op=d.ReduceOp.MAX)
    return t.tolist()


def reduce_sum(values, device=None):
    """Element-wise sum over ranks of a list of floats (identity on one rank)."""
    import torch
    d = _dist()
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if d is not None:
        d.all_reduce(t, op=d.ReduceOp.SUM)
    return t.tolist()


def throughput(units_local: float, seconds_local: float, device=None) -> float:
    """Whole-job units per second: units summed over ranks over the slowest
    rank's time."""
    units = reduce_sum([units_local], device)[0]
    secs = reduce_max([seconds_local], device)[0]
    return units / secs
