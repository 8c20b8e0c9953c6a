"""GPU burn vs the CPU oracle, element by element, through the C ABI.

Every case draws its inputs from the seeded generators (``gen``); expected
values come only from the oracle, and the bar's measured part from the
oracle's own rounding variants on the same zones (``tests/parity.py``).
"""
import numpy as np
import pytest

import gen
import oracle
from tests.parity import compare, oracle_spread, to_numpy

pytestmark = pytest.mark.gpu

_ORACLE = {}


def nb_mod():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2312_02836_gb300 as nb
    return nb, torch


def oracle_run(name, Z, sel=None, **kw):
    """(oracle result, measured spread of its rounding variants) on the
    zones of workload ``name`` (optionally a selection of them)."""
    key = (name, Z, None if sel is None else tuple(sel), tuple(sorted(kw.items())))
    if key not in _ORACLE:
        net, z, s = gen.problem(name, Z)
        if sel is not None:
            z = {k: v[sel] for k, v in z.items()}
        s.update(kw)
        run = lambda v: oracle.burn(net, z["Y"], z["T9"], z["rho"], s["t_end"], s["rtol"],
                                    s["atol"], zeta=z.get("zeta"), variant=v)
        o = run(0)
        _ORACLE[key] = (o, oracle_spread(o, [run(v) for v in oracle.VARIANTS],
                                         s["atol"], s["rtol"]))
    return _ORACLE[key]


def gpu_run(nb, torch, net_c, z, s, **kw):
    dev = torch.device("cuda")
    Y0 = torch.from_numpy(z["Y"]).to(dev)
    T9 = torch.from_numpy(z["T9"]).to(dev)
    rho = torch.from_numpy(z["rho"]).to(dev)
    lm = kw.pop("ln_mult", None)
    if lm is not None:
        lm = torch.from_numpy(np.ascontiguousarray(lm)).to(dev)
    if "zeta" in z:
        kw["zeta"] = torch.from_numpy(z["zeta"]).to(dev)
    out = nb.burn(net_c, Y0, T9, rho, s["t_end"], s["rtol"], s["atol"], lm, **kw)
    torch.cuda.synchronize()
    return to_numpy(out)


CASES = [("chain13", 4096), ("chain13_literal", 1024), ("chain13_heat", 2048),
         ("chain13_heat_ap", 2048), ("chain13_heat_scr", 2048), ("chain13_heat_tab", 2048),
         ("net48", 256), ("net48_adjoint", 128), ("net128_heat", 16)]


# "persistent": the default persistent launch (the network-specialised kernel
# where the network qualifies); "generic": the persistent launch forced onto
# the generic kernel; "plain": one thread per zone; "coop": one warp per zone;
# "coop3": one warp per zone in the variant built for three blocks per SM;
# "team2", "team4": a block of two or four warps per zone
KERNELS = {"persistent": dict(kernel="persistent"),
           "generic": dict(kernel="persistent", specialize="generic"),
           "plain": dict(kernel="plain"),
           "coop": dict(kernel="coop"),
           "coop3": dict(kernel="coop", threads_per_block=32, blocks_per_sm=3),
           "team2": dict(kernel="coop", warps_per_zone=2),
           "team4": dict(kernel="coop", warps_per_zone=4)}


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("name,Z", CASES)
def test_parity_with_oracle(name, Z, kernel):
    nb, torch = nb_mod()
    net, z, s = gen.problem(name, Z)
    net_c = nb.Network(net)
    g = gpu_run(nb, torch, net_c, z, s, **KERNELS[kernel])
    o, spread = oracle_run(name, Z)
    rep = compare(g, o, s["atol"], rtol=s["rtol"], spread=spread)
    if name != "chain13_literal":
        # sum A_i Y_i = 1, except on zones whose outcome the oracle's own
        # rounding variants change (runaway zones, rates ~1e80)
        mass = (g["Y"] * net.A).sum(1)
        ok = g["status"] == 0
        ok[rep["rounding_decided_zones"]] = False
        assert np.abs(mass[ok] - 1.0).max() <= 1e-12
    # no abundance below -atol, on the zones whose outcome is not decided by
    # rounding (a runaway zone that stopped with a failure status keeps its
    # last iterate)
    ok = g["status"] == 0
    ok[rep["rounding_decided_zones"]] = False
    assert g["Y"][ok].min() >= -s["atol"]
    print(name, kernel, rep)


def test_full_size_self_heating_sampled():
    # the benchmark's workload and launch configuration, checked on a seeded
    # sample of zones the oracle can burn one by one
    nb, torch = nb_mod()
    name = "chain13_heat"
    net, z, s = gen.problem(name)
    g = gpu_run(nb, torch, nb.Network(net), z, s)
    Z = z["T9"].shape[0]
    sel = np.unique(np.concatenate([np.arange(64), np.random.default_rng(7).choice(Z, 448, replace=False)]))
    o, spread = oracle_run(name, Z, sel=sel)
    rep = compare({k: v[sel] for k, v in g.items()}, o, s["atol"], spread=spread)
    assert (g["status"] == 0).all()
    print(rep)


def test_edge_cases():
    nb, torch = nb_mod()
    net, z, s = gen.problem("chain13_heat", 37)          # ragged: 37 zones
    net_c = nb.Network(net)
    for kernel in ("persistent", "plain"):
        g = gpu_run(nb, torch, net_c, z, s, kernel=kernel)
        o37, sp37 = oracle_run("chain13_heat", 37)
        compare(g, o37, s["atol"], spread=sp37)
    # Z = 0 and Z = 1
    z0 = {k: v[:0] for k, v in z.items()}
    g0 = gpu_run(nb, torch, net_c, z0, s)
    assert g0["Y"].shape == (0, 13)
    z1 = {k: v[:1] for k, v in z.items()}
    o1, sp1 = oracle_run("chain13_heat", 37, sel=[0])
    compare(gpu_run(nb, torch, net_c, z1, s), o1, s["atol"], spread=sp1)
    # t_end = 0: nothing moves
    s0 = dict(s, t_end=0.0)
    g = gpu_run(nb, torch, net_c, z, s0)
    assert np.array_equal(g["Y"], z["Y"]) and (g["status"] == 0).all()
    assert (g["counters"][:, 0] == 0).all()
    # a non-finite zone is flagged, the others are untouched by it
    zb = {k: v.copy() for k, v in z.items()}
    zb["T9"][5] = np.nan
    zb["Y"][9, 3] = np.inf
    g = gpu_run(nb, torch, net_c, zb, s)
    assert g["status"][5] == 5 and g["status"][9] == 5
    keep = np.setdiff1d(np.arange(37), [5, 9])
    full = gpu_run(nb, torch, net_c, z, s)
    assert np.array_equal(g["Y"][keep], full["Y"][keep])


def test_no_reactions_and_one_body_network():
    nb, torch = nb_mod()
    spec = gen.NetworkSpec(name="empty", N=3, R=0,
                           reactants=np.zeros((0, 3), np.int16),
                           products=np.zeros((0, 3), np.int16),
                           A=np.ones(3), coeffs=np.zeros((0, 7)))
    z = {"Y": np.array([[0.1, 0.2, 0.3]] * 5), "T9": np.full(5, 2.0), "rho": np.full(5, 1e6)}
    s = dict(t_end=1.0, rtol=1e-8, atol=1e-12)
    g = gpu_run(nb, torch, nb.Network(spec), z, s)
    # f = 0: the BDF formula reproduces x up to rounding of sum_j alpha_j = 0
    np.testing.assert_allclose(g["Y"], z["Y"], rtol=1e-13, atol=0)
    assert (g["status"] == 0).all()


def test_deterministic_and_order_independent():
    nb, torch = nb_mod()
    net, z, s = gen.problem("chain13_heat", 1000)
    net_c = nb.Network(net)
    a = gpu_run(nb, torch, net_c, z, s)
    b = gpu_run(nb, torch, net_c, z, s)
    for k in a:
        assert np.array_equal(a[k], b[k])
    perm = np.random.default_rng(1).permutation(1000)
    zp = {k: v[perm] for k, v in z.items()}
    c = gpu_run(nb, torch, net_c, zp, s)
    for k in a:
        assert np.array_equal(a[k][perm], c[k])
    # launch shape and blob placement do not change any bit
    d = gpu_run(nb, torch, net_c, z, s, threads_per_block=64, blocks_per_sm=1,
                blob_in_shared=0)
    e = gpu_run(nb, torch, net_c, z, s, kernel="plain")
    f = gpu_run(nb, torch, net_c, z, s, threads_per_block=224, ws_in_shared=3)
    g = gpu_run(nb, torch, net_c, z, s, threads_per_block=96, ws_in_shared=3,
                blocks_per_sm=2)
    for k in a:
        for other in (d, e, f, g):
            assert np.array_equal(a[k], other[k])
    # the warp-per-zone kernel: deterministic, independent of the claim order
    # and of where its arrays live (its solves and sums round differently from
    # the lane kernels', so it is compared with the oracle elsewhere)
    c1 = gpu_run(nb, torch, net_c, z, s, kernel="coop")
    c2 = gpu_run(nb, torch, net_c, zp, s, kernel="coop", threads_per_block=64)
    c3 = gpu_run(nb, torch, net_c, z, s, kernel="coop", ws_in_shared=0, blob_in_shared=0)
    for k in a:
        assert np.array_equal(c1[k][perm], c2[k])
        assert np.array_equal(c1[k], c3[k])


def test_rate_multipliers_shared_and_per_zone():
    nb, torch = nb_mod()
    net, z, s = gen.problem("net48", 64)
    net_c = nb.Network(net)
    lm = np.random.default_rng(3).normal(0.0, 0.5, net.R)
    a = gpu_run(nb, torch, net_c, z, s, ln_mult=lm)
    b = gpu_run(nb, torch, net_c, z, s, ln_mult=np.tile(lm, (64, 1)))
    for k in a:
        assert np.array_equal(a[k], b[k])
    run = lambda v: oracle.burn(net, z["Y"], z["T9"], z["rho"], s["t_end"], s["rtol"],
                                s["atol"], ln_mult=lm, variant=v)
    o = run(0)
    compare(a, o, s["atol"], variants=[run(v) for v in oracle.VARIANTS])


def test_host_entry_point_matches_device_entry_point():
    nb, torch = nb_mod()
    net, z, s = gen.problem("chain13_heat", 300)
    net_c = nb.Network(net)
    a = gpu_run(nb, torch, net_c, z, s)
    h = nb.burn_host(net_c, z["Y"], z["T9"], z["rho"], s["t_end"], s["rtol"], s["atol"])
    for k in a:
        assert np.array_equal(a[k], h[k])


def test_operator_split_per_zone_end_times():
    # every zone burns for its own hydro step (log-uniform 1e-6 .. 1e-3 s)
    nb, torch = nb_mod()
    net, z, s = gen.problem("chain13_heat", 1500)
    tz = np.exp(np.random.default_rng(21).uniform(np.log(1e-6), np.log(1e-3), 1500))
    tz[7] = np.nan
    tz[8] = -1.0
    dev = torch.device("cuda")
    g = nb.burn(nb.Network(net), torch.from_numpy(z["Y"]).to(dev),
                torch.from_numpy(z["T9"]).to(dev), torch.from_numpy(z["rho"]).to(dev),
                torch.from_numpy(tz).to(dev), s["rtol"], s["atol"])
    torch.cuda.synchronize()
    g = to_numpy(g)
    run = lambda v: oracle.burn(net, z["Y"], z["T9"], z["rho"], tz, s["rtol"], s["atol"],
                                variant=v)
    o = run(0)
    assert g["status"][7] == 5 and g["status"][8] == 5
    print(compare(g, o, s["atol"], variants=[run(v) for v in oracle.VARIANTS]))
