"""Several networks in one launch (nb_burn_multi): every set's zones must
come out bit for bit as a single-network burn of the same zones gives them
(the generic kernel, and so the specialised one too), whatever sets share
the launch; and each set's zones meet the parity bar against the oracle
directly."""
import numpy as np
import pytest

import gen
import oracle
from tests.parity import compare, oracle_spread, to_numpy

pytestmark = pytest.mark.gpu


def _mods():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2312_02836_gb300 as nb
    return nb, torch


def _set(nb, torch, name, Z, **extra):
    net, z, s = gen.problem(name, Z)
    t = {k: torch.from_numpy(v).cuda() for k, v in z.items()}
    d = dict(net=nb.Network(net), Y0=t["Y"], T9=t["T9"], rho=t["rho"], **extra)
    return d, net, s


def _equal(a, b):
    import torch
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_multi_network_batch_equals_single_burns():
    nb, torch = _mods()
    sets, specs = [], []
    for name, Z in (("chain13_heat", 1024), ("net48", 96), ("chain13", 512),
                    ("chain13_literal", 200)):
        d, net, s = _set(nb, torch, name, Z)
        sets.append(d)
        specs.append(s)
    # every workload here shares t_end, rtol, atol except net48 (t_end 1e-2):
    # burn the whole batch at one t_end, overriding net48's per zone
    s0 = specs[0]
    tz = torch.full((96,), specs[1]["t_end"], dtype=torch.float64, device="cuda")
    sets[1]["t_end"] = tz
    outs = nb.burn_multi(sets, s0["t_end"], s0["rtol"], s0["atol"])
    torch.cuda.synchronize()
    for d, s, out in zip(sets, specs, outs):
        te = d.get("t_end", s0["t_end"])
        ref = nb.burn(d["net"], d["Y0"], d["T9"], d["rho"], te, s0["rtol"], s0["atol"],
                      specialize="generic")
        torch.cuda.synchronize()
        assert int((out.status == 0).sum()) == d["Y0"].shape[0]
        _equal(out, ref)


def test_multi_network_options_and_empty_set():
    nb, torch = _mods()
    a, _, s = _set(nb, torch, "chain13_heat", 300)
    b, net_b, _ = _set(nb, torch, "chain13", 0)
    rng = np.random.default_rng(3)
    lm = torch.from_numpy(rng.normal(0.0, 0.2, (300, a["net"].R))).cuda()
    a["ln_mult"] = lm
    outs = nb.burn_multi([b, a], s["t_end"], s["rtol"], s["atol"], threads_per_block=64,
                         blocks_per_sm=2)
    torch.cuda.synchronize()
    assert outs[0].Y.shape[0] == 0
    ref = nb.burn(a["net"], a["Y0"], a["T9"], a["rho"], s["t_end"], s["rtol"], s["atol"],
                  lm, specialize="generic")
    torch.cuda.synchronize()
    _equal(outs[1], ref)
    # argument errors are caught on the host
    with pytest.raises(nb.NetburnError):
        nb.burn_multi([a] * 13, s["t_end"], s["rtol"], s["atol"])
    with pytest.raises(nb.NetburnError):
        nb.burn_multi([a], s["t_end"], -1.0, s["atol"])


def test_multi_network_batch_with_screening_and_tables():
    # screened (per-set plasma parameters), tabulated and effective-rate
    # networks in one launch: each set as its single-network burn
    nb, torch = _mods()
    sets, specs = [], []
    for name, Z in (("chain13_heat_scr", 300), ("chain13_heat_tab", 300),
                    ("chain13_heat_ap", 200)):
        net, z, s = gen.problem(name, Z)
        t = {k: torch.from_numpy(v).cuda() for k, v in z.items()}
        d = dict(net=nb.Network(net), Y0=t["Y"], T9=t["T9"], rho=t["rho"])
        if "zeta" in t:
            d["zeta"] = t["zeta"]
        sets.append(d)
        specs.append(s)
    s0 = specs[0]
    outs = nb.burn_multi(sets, s0["t_end"], s0["rtol"], s0["atol"])
    torch.cuda.synchronize()
    for d, out in zip(sets, outs):
        ref = nb.burn(d["net"], d["Y0"], d["T9"], d["rho"], s0["t_end"], s0["rtol"],
                      s0["atol"], specialize="generic", zeta=d.get("zeta"))
        torch.cuda.synchronize()
        assert int((out.status == 0).sum()) == d["Y0"].shape[0]
        _equal(out, ref)


def test_multi_network_batch_against_oracle():
    # one launch over four networks (fixed T, self-heating, screened, 48
    # species at its own end time per zone), each set held to the oracle
    nb, torch = _mods()
    cases = (("chain13_heat", 512), ("net48", 64), ("chain13", 256), ("chain13_heat_scr", 256))
    sets, probs = [], []
    for name, Z in cases:
        d, net, s = _set(nb, torch, name, Z)
        z = gen.problem(name, Z)[1]
        if "zeta" in z:
            d["zeta"] = torch.from_numpy(z["zeta"]).cuda()
        sets.append(d)
        probs.append((net, z, s))
    s0 = probs[0][2]
    for d, (net, z, s) in zip(sets, probs):
        assert (s["rtol"], s["atol"]) == (s0["rtol"], s0["atol"])
        if s["t_end"] != s0["t_end"]:
            d["t_end"] = torch.full((z["T9"].shape[0],), s["t_end"], dtype=torch.float64,
                                    device="cuda")
    outs = nb.burn_multi(sets, s0["t_end"], s0["rtol"], s0["atol"])
    torch.cuda.synchronize()
    for (name, Z), (net, z, s), out in zip(cases, probs, outs):
        run = lambda v: oracle.burn(net, z["Y"], z["T9"], z["rho"], s["t_end"], s["rtol"],
                                    s["atol"], zeta=z.get("zeta"), variant=v)
        o = run(0)
        spread = oracle_spread(o, [run(v) for v in oracle.VARIANTS], s["atol"], s["rtol"])
        rep = compare(to_numpy(out), o, s["atol"], rtol=s["rtol"], spread=spread)
        assert (to_numpy(out)["status"] == 0).all()
        print(name, rep)
