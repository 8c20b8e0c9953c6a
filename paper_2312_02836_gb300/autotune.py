"""Launch-shape autotuner for the persistent burn kernels.

The tunables are which kernel runs (one zone per lane, generic or generated
for the network, or one zone per warp), how many zones are in flight per SM
and where their work arrays live:

* ``specialize``: -1 the generic kernel, which walks the compiled network
  from memory; 1..3 the kernel generated for this network, with its work
  arrays in registers (1), the LU in the workspace (2) or only x, d, f in
  registers (3).  Specialised candidates are tried only for networks the
  library would specialise by itself (their straight-line code compiles in
  seconds);
* ``ws_in_shared`` w (generic kernel): the first w warps of each block keep
  their Newton-loop arrays in shared memory (history in global memory), the
  others keep everything in the global workspace, which stays L2-resident
  only while few lanes are in flight;
* ``threads_per_block`` and ``blocks_per_sm``: zones in flight.  Fewer lanes
  than zones let the device queue refill lanes whose zone finished; more
  lanes hide more latency but grow the workspace beyond L2;
* ``kernel="coop"`` (networks of 24 or more state entries): one warp per
  zone with its Newton-loop arrays in shared memory; threads_per_block sets
  the warps per block, hence the zones per SM that share its memory.

Each candidate burns the caller's zones once and is timed with CUDA events
on the current stream; the fastest wins.  Results are cached per network,
device and zone count for the life of the process.
"""
from __future__ import annotations

from typing import Optional

_CACHE: dict = {}

GENERIC_CANDIDATES = (
    dict(specialize=-1, ws_in_shared=0, threads_per_block=128, blocks_per_sm=1),
    dict(specialize=-1, ws_in_shared=1, threads_per_block=160, blocks_per_sm=1),
    dict(specialize=-1, ws_in_shared=3, threads_per_block=96, blocks_per_sm=1),
    dict(specialize=-1, ws_in_shared=0, threads_per_block=64, blocks_per_sm=2),
    dict(specialize=-1, ws_in_shared=0, threads_per_block=128, blocks_per_sm=2),
)

SPECIALIZED_CANDIDATES = tuple(
    dict(specialize=v, threads_per_block=tpb, blocks_per_sm=bps)
    for v in (1, 2, 3) for tpb, bps in ((64, 1), (128, 1), (128, 2), (256, 1)))

# one warp per zone, its Newton-loop arrays in shared memory (large networks)
COOP_CANDIDATES = (
    dict(kernel="coop", threads_per_block=0, blocks_per_sm=0),
    dict(kernel="coop", threads_per_block=64, blocks_per_sm=0),
    dict(kernel="coop", threads_per_block=32, blocks_per_sm=0),
    # one block of four warps per SM: less shared memory taken, more L1 left
    # for the network's index lists
    dict(kernel="coop", threads_per_block=128, blocks_per_sm=1),
    # three blocks of four warps per SM (registers capped, some spilled),
    # where their shared-memory arrays fit
    dict(kernel="coop", threads_per_block=128, blocks_per_sm=3),
    # the same claiming zones in index order: with many zones per warp the
    # longest-first pre-pass costs more than it saves (48 species: 6.94 s
    # against 7.80 s at 262,144 zones, 0.60 s against 0.53 s at 16,384)
    dict(kernel="coop", threads_per_block=128, blocks_per_sm=3, schedule="fifo"),
    # a block of two or four warps per zone: more lanes on each zone's LU
    # where the arrays of one zone take much of an SM's shared memory
    dict(kernel="coop", warps_per_zone=2),
    dict(kernel="coop", warps_per_zone=4),
)

DEFAULT_CANDIDATES = GENERIC_CANDIDATES + SPECIALIZED_CANDIDATES + COOP_CANDIDATES


def eligible(info: dict, candidates=DEFAULT_CANDIDATES) -> list:
    """The candidates worth timing for a network (``Network.info()``)."""
    out = list(candidates)
    if not info["specialize_auto"]:
        # no generated kernel for this network: the generic and warp kernels
        out = [c for c in out if c.get("kernel") == "coop" or c.get("specialize", 0) < 0]
    if info["n_state"] < 24:
        # a warp per zone leaves most lanes idle on a small network
        out = [c for c in out if c.get("kernel") != "coop"]
    return out


def autotune(net, Y0, T9, rho, t_end, rtol, atol, ln_mult=None, *,
             candidates=DEFAULT_CANDIDATES, key: Optional[str] = None,
             verbose: bool = False, extra: Optional[dict] = None) -> dict:
    """Return the fastest launch options for burning these zones (extra:
    further keyword arguments of every burn, e.g. the plasma parameters)."""
    extra = extra or {}
    import torch

    from . import NetburnError, burn

    dev = Y0.device
    ck = (key or id(net), torch.cuda.get_device_name(dev), int(Y0.shape[0]))
    if ck in _CACHE:
        return dict(_CACHE[ck])
    stream = torch.cuda.current_stream(dev)
    best, best_ms, timings = None, float("inf"), []
    out = None
    candidates = eligible(net.info(), candidates)
    for cand in candidates:
        try:
            out = burn(net, Y0, T9, rho, t_end, rtol, atol, ln_mult, out=out, **cand, **extra)
        except NetburnError:
            continue                      # does not fit this network / GPU
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        burn(net, Y0, T9, rho, t_end, rtol, atol, ln_mult, out=out, **cand, **extra)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        timings.append((cand, ms))
        if verbose:
            print("autotune", cand, f"{ms:.1f} ms")
        if ms < best_ms:
            best, best_ms = cand, ms
    if best is None:
        raise NetburnError("no launch shape fits this network")
    _CACHE[ck] = dict(best)
    result = dict(best)
    result["_timings_ms"] = [(dict(c), m) for c, m in timings]
    return result
