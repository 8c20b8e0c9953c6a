"""Zone sharding across processes (one process per GPU).

Zones burn independently, so N ranks split the zones into contiguous
ranges and burn them with no collective on the data path.  The ranges can
be balanced by predicted cost (``zone_costs``: the library's start-up
estimate) rather than by count, since zones of a hydro grid differ in
stiffness by orders of magnitude.  The only communication is host-side
bookkeeping: the slowest rank's time (what a job waits for) and, for a rate
gradient shared by all zones, one sum of an R-vector.
"""
from __future__ import annotations


def shard(Z: int, world: int, rank: int, cost=None) -> tuple[int, int]:
    """[begin, end) of rank's contiguous share of Z zones.  Without cost the
    shares differ in size by at most one; with cost (a sequence of Z
    non-negative weights, e.g. ``zone_costs``) each range holds about
    1/world of the total weight: rank r starts at the first zone whose
    preceding weight reaches r/world of the total."""
    if world < 1 or not 0 <= rank < world or Z < 0:
        raise ValueError("bad shard request")
    if cost is None:
        base, extra = divmod(Z, world)
        begin = rank * base + min(rank, extra)
        return begin, begin + base + (1 if rank < extra else 0)
    import numpy as np
    c = np.asarray(cost, dtype=np.float64).reshape(-1)
    if c.size != Z or (c < 0).any() or not np.isfinite(c).all():
        raise ValueError("cost must hold Z finite non-negative weights")
    before = np.concatenate([[0.0], np.cumsum(c)[:-1]])
    total = float(c.sum())
    if total <= 0.0:
        return shard(Z, world, rank)
    edge = lambda r: Z if r >= world else int(np.searchsorted(before, r * total / world, "left"))
    return edge(rank), edge(rank + 1)


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
