"""Multi-process sharding of zones, on CPU with two gloo ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2312_02836_gb300.parallel import max_over_ranks, shard, sum_over_ranks


def test_shard_covers_every_zone_once():
    for Z in (0, 1, 7, 65536, 65537):
        for world in (1, 2, 3, 8):
            ranges = [shard(Z, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == Z
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        Z = 1001
        a, b = shard(Z, world, rank)
        # each rank "burns" its zones (a stand-in: per-zone work time)
        t = float(b - a) * (1.0 + rank)
        tmax = max_over_ranks(t)
        g = torch.full((5,), float(rank + 1), dtype=torch.float64)
        sum_over_ranks(g)
        q.put((rank, a, b, tmax, g.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, a0, b0, m0, g0), (r1, a1, b1, m1, g1) = out
    assert (a0, b1) == (0, 1001) and b0 == a1
    expect_max = max((b0 - a0) * 1.0, (b1 - a1) * 2.0)
    assert m0 == m1 == expect_max
    assert g0 == g1 == [3.0] * 5
