"""The network-specialised kernel (CUDA generated per network, compiled at
run time) against the generic kernel.  Both perform the same floating-point
operations in the same order, so every output must be equal bit for bit,
for every storage variant and every option that changes the integration
(per-zone multipliers, per-zone end times, the adjoint tape).  Parity with
the oracle is checked by the parity tests, which run both kernels."""
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


def _equal(a, b):
    import torch
    for x, y in zip(a, b):
        assert torch.equal(x, y)


CASES = [("chain13", 2048), ("chain13_literal", 1024), ("chain13_heat", 2048),
         ("chain13_heat_ap", 1024), ("chain13_heat_scr", 1024), ("chain13_heat_tab", 1024)]


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("name,Z", CASES)
def test_specialized_equals_generic_bitwise(name, Z, variant):
    nb, torch, net, z, s, t = _setup(name, Z)
    nc = nb.Network(net)
    args = (nc, t["Y"], t["T9"], t["rho"], s["t_end"], s["rtol"], s["atol"])
    zk = dict(zeta=t["zeta"]) if "zeta" in t else {}
    ref = nb.burn(*args, specialize="generic", **zk)
    assert nc.info()["last_specialized"] == 0
    out = nb.burn(*args, specialize=variant, **zk)
    torch.cuda.synchronize()
    assert nc.info()["last_specialized"] == variant
    assert int((out.status == 0).sum()) == Z
    _equal(out, ref)
    # other launch shapes of the specialised kernel: the same bits
    for tpb, bps in ((64, 1), (128, 2), (256, 1)):
        again = nb.burn(*args, specialize=variant, threads_per_block=tpb,
                        blocks_per_sm=bps, schedule="fifo", **zk)
        torch.cuda.synchronize()
        _equal(again, ref)


def test_automatic_choice():
    nb, torch, net, z, s, t = _setup("chain13_heat", 512)
    nc = nb.Network(net)
    info = nc.info()
    assert info["specialize_auto"] == 1
    nb.burn(nc, t["Y"], t["T9"], t["rho"], s["t_end"], s["rtol"], s["atol"])
    torch.cuda.synchronize()
    assert nc.info()["last_specialized"] in (1, 2, 3)
    nb.burn(nc, t["Y"], t["T9"], t["rho"], s["t_end"], s["rtol"], s["atol"],
            kernel="plain")
    assert nc.info()["last_specialized"] == 0
    # a network too large for straight-line code stays on the generic kernel
    big = nb.Network(gen.network("net128_heat"))
    assert big.info()["specialize_auto"] == 0
    log = nc.specialize(3)
    assert "error" not in log.lower()


def test_specialized_options_and_tape_bitwise():
    # per-zone rate multipliers, per-zone end times and the recorded tape:
    # the adjoint of the two tapes must agree to the bit as well
    name, Z = "chain13_heat", 1024
    nb, torch, net, z, s, t = _setup(name, Z)
    nc = nb.Network(net)
    rng = np.random.default_rng(7)
    lm = torch.from_numpy(rng.normal(0.0, 0.3, (Z, net.R))).cuda()
    tz = torch.from_numpy(s["t_end"] * rng.uniform(0.1, 1.0, Z)).cuda()
    outs, grads = [], []
    for sp in ("generic", 2):
        tape = nb.Tape(nc, Z, 4000)
        out = nb.burn(nc, t["Y"], t["T9"], t["rho"], tz, s["rtol"], s["atol"], lm,
                      tape=tape, specialize=sp)
        torch.cuda.synchronize()
        assert int((out.status == 0).sum()) == Z
        gY = torch.zeros((1, Z, net.N), dtype=torch.float64, device="cuda")
        gY[0, :, 3] = 1.0
        gE = torch.ones((1, Z), dtype=torch.float64, device="cuda")
        g = nb.adjoint(nc, tape, gY, gE)
        torch.cuda.synchronize()
        outs.append(out)
        grads.append(g)
    _equal(outs[0], outs[1])
    for a, b in zip(grads[0], grads[1]):
        if a is not None:
            assert torch.equal(a, b)


def test_specialized_watchdog():
    # the watchdog lives in the shared claim loop: an exhausted budget ends
    # zones with TIMEOUT in the specialised kernel too
    nb, torch, net, z, s, t = _setup("chain13_heat", 4096)
    nc = nb.Network(net)
    out = nb.burn(nc, t["Y"], t["T9"], t["rho"], s["t_end"], s["rtol"], s["atol"],
                  specialize=1, time_budget_s=1e-9)
    torch.cuda.synchronize()
    st = out.status.cpu().numpy()
    assert (st == 6).sum() > 0
    done = st == 0
    ref = nb.burn(nc, t["Y"], t["T9"], t["rho"], s["t_end"], s["rtol"], s["atol"],
                  specialize="generic")
    torch.cuda.synchronize()
    assert torch.equal(out.Y[torch.from_numpy(done).cuda()],
                       ref.Y[torch.from_numpy(done).cuda()])
