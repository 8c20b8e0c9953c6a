"""Runtime features of the burn on the GPU: CUDA-graph replay and the
device watchdog (a time budget that ends zones with TIMEOUT instead of
letting a call run on)."""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


def _setup(name, Z):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2312_02836_gb300 as nb
    net, z, s = gen.problem(name, Z)
    dev = torch.device("cuda")
    t = {k: torch.from_numpy(v).to(dev) for k, v in z.items()}
    return nb, torch, net, z, s, t


def test_graph_replay_matches_direct_burn():
    nb, torch, net, z, s, t = _setup("chain13_heat", 2000)
    nc = nb.Network(net)
    g = nb.BurnGraph(nc, t["Y"], t["T9"], t["rho"], s["t_end"], s["rtol"], s["atol"])
    ref = nb.burn(nc, t["Y"], t["T9"], t["rho"], s["t_end"], s["rtol"], s["atol"])
    out = g.replay()
    torch.cuda.synchronize()
    for a, b in zip(out, ref):
        assert torch.equal(a, b)
    # new inputs written in place, replayed
    z2 = gen.zones("chain13_heat", 4000)
    t["T9"].copy_(torch.from_numpy(z2["T9"][2000:]))
    t["rho"].copy_(torch.from_numpy(z2["rho"][2000:]))
    out = g.replay()
    ref2 = nb.burn(nc, t["Y"], t["T9"], t["rho"], s["t_end"], s["rtol"], s["atol"])
    torch.cuda.synchronize()
    for a, b in zip(out, ref2):
        assert torch.equal(a, b)


@pytest.mark.parametrize("kernel", ["persistent", "plain"])
def test_watchdog_ends_zones_with_timeout(kernel):
    nb, torch, net, z, s, t = _setup("chain13_heat", 20000)
    nc = nb.Network(net)
    full = nb.burn(nc, t["Y"], t["T9"], t["rho"], s["t_end"], s["rtol"], s["atol"],
                   kernel=kernel)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    cut = nb.burn(nc, t["Y"], t["T9"], t["rho"], s["t_end"], s["rtol"], s["atol"],
                  kernel=kernel, time_budget_s=2e-3)
    b.record()
    torch.cuda.synchronize()
    st = cut.status.cpu().numpy()
    assert set(np.unique(st)) <= {0, 6}
    assert (st == 6).sum() > 0
    assert a.elapsed_time(b) < 0.5 * 1e3          # well under a normal burn
    ok = st == 0
    assert np.array_equal(cut.Y.cpu().numpy()[ok], full.Y.cpu().numpy()[ok])
    # a timed-out zone holds the state it reached: finite, and mass conserved
    Yc = cut.Y.cpu().numpy()[~ok]
    assert np.isfinite(Yc).all()
    assert np.abs((Yc * net.A).sum(1) - 1.0).max() <= 1e-12
    # the context is usable afterwards
    again = nb.burn(nc, t["Y"], t["T9"], t["rho"], s["t_end"], s["rtol"], s["atol"],
                    kernel=kernel)
    torch.cuda.synchronize()
    assert torch.equal(again.Y, full.Y)
