"""Zone sharding across processes (one process per GPU).

Zones burn independently, so N ranks split the zones into contiguous
ranges and burn them with no collective on the data path.  The only
communication is host-side bookkeeping: the slowest rank's time (what a
job waits for) and, for a rate gradient shared by all zones, one sum of an
R-vector.
"""
from __future__ import annotations


def shard(Z: int, world: int, rank: int) -> tuple[int, int]:
    """[begin, end) of rank's contiguous share of Z zones (sizes differ by
    at most one)."""
    if world < 1 or not 0 <= rank < world or Z < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(Z, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a scalar over the default process group (identity when
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(tensor):
    """In-place sum of a tensor over the default process group (e.g. the
    gradient with respect to rate multipliers shared by every zone)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(tensor, op=dist.ReduceOp.SUM)
    return tensor
