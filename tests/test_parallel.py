"""Multi-process sharding of zones, on CPU with two gloo ranks.

The GPU path shards zones across ranks with no collective on the data
path; each rank's burn is the library's single-GPU burn.  Here the ranks
burn their shares with the CPU oracle (the same per-zone map), so the test
checks the sharding, the balance by predicted cost, the gathering and the
timing bookkeeping end to end, without a GPU."""
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


def test_shard_by_cost_balances_weight():
    rng = np.random.default_rng(3)
    for Z, world in ((1000, 2), (4097, 8), (10, 3)):
        cost = rng.lognormal(0.0, 2.0, Z)
        ranges = [shard(Z, world, r, cost) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == Z
        assert all(b == c for (a, b), (c, d) in zip(ranges, ranges[1:]))
        w = np.array([cost[a:b].sum() for a, b in ranges])
        # each range holds its share to within the heaviest single zone
        assert np.abs(w - cost.sum() / world).max() <= cost.max() + 1e-9
    # all weight in one zone: rank 1 starts after it (its weight is what
    # precedes zone 7), so rank 0 takes zones 0..6
    c = np.zeros(10)
    c[6] = 1.0
    assert shard(10, 2, 0, c) == (0, 7) and shard(10, 2, 1, c) == (7, 10)
    assert shard(5, 2, 0, np.zeros(5)) == shard(5, 2, 0)
    with pytest.raises(ValueError):
        shard(3, 2, 0, [1.0, -1.0, 2.0])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _costs(net, z, s):
    """(1 + ln(t_end / h0))^2 per zone, h0 the oracle's starting step (the
    quantity nb_zone_costs computes on the GPU)."""
    import oracle
    out = []
    for i in range(z["T9"].shape[0]):
        tp = oracle.burn_tape(net, z["Y"][i], z["T9"][i], z["rho"][i], s["t_end"], s["rtol"],
                              s["atol"], max_attempts=1)
        h0 = tp["t"][-1]
        out.append(0.0 if h0 <= 0 else (1.0 + max(np.log(s["t_end"] / h0), 0.0)) ** 2)
    return np.array(out)


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import time

        import gen
        import oracle
        Z = 96
        net, z, s = gen.problem("net48", Z)
        cost = _costs(net, z, s)
        a, b = shard(Z, world, rank, cost)
        t0 = time.perf_counter()
        part = oracle.burn(net, z["Y"][a:b], z["T9"][a:b], z["rho"][a:b], s["t_end"], s["rtol"],
                           s["atol"], threads=1)
        tmax = max_over_ranks(time.perf_counter() - t0)
        # gather every rank's zones (padded to the largest share)
        n = torch.tensor([b - a])
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, n)
        m = max(int(v) for v in sizes)
        mine = torch.zeros((m, net.N), dtype=torch.float64)
        mine[:b - a] = torch.from_numpy(part["Y"])
        allY = [torch.zeros((m, net.N), dtype=torch.float64) for _ in range(world)]
        dist.all_gather(allY, mine)
        Y = np.concatenate([allY[r][:int(sizes[r])].numpy() for r in range(world)])
        attempts = torch.tensor([float(part["counters"][:, :3].sum())], dtype=torch.float64)
        per_rank = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(per_rank, attempts)
        g = torch.full((5,), float(rank + 1), dtype=torch.float64)
        sum_over_ranks(g)
        q.put((rank, a, b, tmax, g.tolist(), Y, [float(v) for v in per_rank],
               float(cost[a:b].sum()), float(cost.sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_burn_cost_balanced_shards():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, a0, b0, m0, g0, Y0, att0, c0, ctot), (r1, a1, b1, m1, g1, Y1, att1, c1, _) = out
    assert (a0, b1) == (0, 96) and b0 == a1
    assert m0 == m1
    assert g0 == g1 == [3.0] * 5
    # the gathered burn is the single-process burn, bit for bit
    import gen
    import oracle
    net, z, s = gen.problem("net48", 96)
    full = oracle.burn(net, z["Y"], z["T9"], z["rho"], s["t_end"], s["rtol"], s["atol"])
    assert np.array_equal(Y0, full["Y"]) and np.array_equal(Y1, full["Y"])
    # the predicted cost is split evenly; the work it predicts is closer to
    # even than with equal zone counts
    assert abs(c0 - c1) <= 0.2 * ctot
    att = full["counters"][:, :3].sum(1)
    h = 96 // 2
    by_count = abs(att[:h].sum() - att[h:].sum())
    by_cost = abs(att0[0] - att0[1])
    assert by_cost < by_count
