"""GPU discrete adjoint vs the oracle's forward sensitivity of the same
discrete map (frozen schedule, exact Newton solutions), through the C ABI
and through the autograd Function."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


def nb_mod():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2312_02836_gb300 as nb
    return nb, torch


def _forward_sens(net, z, s, zones, ln_mult=None):
    """Oracle (dx/dtheta, dE/dtheta, accepted steps) per zone."""
    out = []
    for i in zones:
        lm = None if ln_mult is None else ln_mult
        zeta = float(z["zeta"][i]) if "zeta" in z else 0.0
        tp = oracle.burn_tape(net, z["Y"][i], z["T9"][i], z["rho"][i], s["t_end"],
                              s["rtol"], s["atol"], ln_mult=lm, zeta=zeta)
        assert tp["status"] == 0
        dx, dE = oracle.forward_sensitivity(net, z["T9"][i], z["rho"][i], tp["t"],
                                            tp["k"], tp["x"], ln_mult=lm, zeta=zeta)
        out.append((dx, dE, int(tp["counters"][0])))
    return out


def _gpu_adjoint(nb, torch, net, z, s, gY, gE, gT9, ln_mult=None, max_steps=20000):
    dev = torch.device("cuda")
    Z = z["T9"].shape[0]
    nc = nb.Network(net)
    tape = nb.Tape(nc, Z, max_steps)
    lm = None if ln_mult is None else torch.from_numpy(ln_mult).to(dev)
    fw = nb.burn(nc, torch.from_numpy(z["Y"]).to(dev), torch.from_numpy(z["T9"]).to(dev),
                 torch.from_numpy(z["rho"]).to(dev), s["t_end"], s["rtol"], s["atol"], lm,
                 tape=tape, zeta=torch.from_numpy(z["zeta"]).to(dev) if "zeta" in z else None)
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    dl, dY0, dT0 = nb.adjoint(nc, tape, t(gY), t(gE), t(gT9))
    torch.cuda.synchronize()
    return (dl.cpu().numpy(), dY0.cpu().numpy(), dT0.cpu().numpy(),
            fw.counters.cpu().numpy(), fw.Y.cpu().numpy(), fw.status.cpu().numpy())


def _check(expect, got, rtol, scale=None, out_mag=0.0, abs_floor=0.0):
    # Entries far below the gradient's scale come from cancelling sums that
    # the two methods accumulate in different orders; a gradient of an
    # output O is known to ~1e-13 |O| absolute (rounding over ~10^3 steps).
    scale = (np.abs(expect).max() if scale is None else scale) + 1e-300
    err = np.abs(got - expect)
    bad = err > rtol * np.abs(expect) + 1e-8 * scale + 1e-13 * out_mag + abs_floor
    assert not bad.any(), (np.where(bad), got[bad][:4], expect[bad][:4])


@pytest.mark.parametrize("name,Z", [("net48_adjoint", 24), ("chain13_heat", 48),
                                    ("chain13_heat_scr", 32), ("chain13_heat_ap", 24)])
def test_adjoint_matches_forward_sensitivity(name, Z):
    nb, torch = nb_mod()
    net, z, s = gen.problem(name, Z)
    n = net.N + (1 if net.self_heating else 0)
    # cotangents: E, and the 5 largest final abundances of each zone (one-hot)
    o = oracle.burn(net, z["Y"], z["T9"], z["rho"], s["t_end"], s["rtol"], s["atol"],
                    zeta=z.get("zeta"))
    top = gen.largest_species(o["Y"], 5)
    K = 6
    gY = np.zeros((K, Z, net.N))
    gE = np.zeros((K, Z))
    gE[0] = 1.0
    for q in range(5):
        gY[q + 1, np.arange(Z), top[:, q]] = 1.0
    gT9 = np.zeros((K, Z)) if net.self_heating else None
    dl, dY0, dT0, cnt, Yf, st = _gpu_adjoint(nb, torch, net, z, s, gY, gE, gT9)
    assert (st == 0).all()
    sens = _forward_sens(net, z, s, range(Z))
    same = 0
    for i, (dx, dE, acc) in enumerate(sens):
        if acc != cnt[i, 0]:
            continue          # a different step sequence is a different map
        same += 1
        for q in range(K):
            w = gY[q, i]
            mag = np.abs(w) @ np.abs(Yf[i]) + abs(gE[q, i]) * abs(o["E"][i])
            # Newton leaves every state entry within 1e-3 of its weight
            # atol + rtol|Y| (C6), so the linearisation point of the frozen
            # map - and the sensitivity of an output Y - is known to about
            # 1e-3 w / |Y| relative; negligible unless Y is near atol
            # 1e-6: the GPU and the oracle linearise along trajectories that
            # differ at the rounding level, and long stiff zones amplify that
            # (one 868-step zone's energy gradient differs by 3e-7 between the
            # oracle built on x86-64 and on aarch64, whose libm differ)
            rt = 1e-6
            floor = 0.0
            if q > 0:
                y = abs(Yf[i][top[i, q - 1]])
                wy = s["atol"] + s["rtol"] * y
                rt += 1e-3 * wy / max(y, 1e-300)
                if y < 1e3 * s["atol"]:
                    # an output below ~1e3 atol is resolved by the method only
                    # to about its weight (error test: w; Newton: 1e-3 w per
                    # step, accumulated): its gradient is held to 1e-2 w
                    floor = 1e-2 * wy
            exp_l = w @ dx[:net.N, :net.R] + gE[q, i] * dE[:net.R]
            _check(exp_l, dl[q, i], rt, out_mag=mag, abs_floor=floor)
            exp_y0 = w @ dx[:net.N, net.R:net.R + net.N] + gE[q, i] * dE[net.R:net.R + net.N]
            _check(exp_y0, dY0[q, i], rt, out_mag=mag, abs_floor=floor)
            col = net.R + net.N   # T9: initial state entry or parameter
            exp_t = w @ dx[:net.N, col] + gE[q, i] * dE[col]
            _check(np.array([exp_t]), np.array([dT0[q, i]]), rt,
                   scale=np.abs(exp_y0).max() * max(1.0, abs(z["T9"][i])), abs_floor=floor)
    assert same >= 0.9 * Z


@pytest.mark.parametrize("name,zone", [("net48_adjoint", 2), ("chain13_heat", 0)])
def test_adjoint_against_frozen_schedule_central_differences(name, zone):
    # central differences of the exactly converged (full-Newton) frozen map,
    # on the oracle's schedule; checked where the GPU took as many steps
    nb, torch = nb_mod()
    net, z, s = gen.problem(name, zone + 1)
    zz = {k: v[zone:zone + 1] for k, v in z.items()}
    tp = oracle.burn_tape(net, zz["Y"][0], zz["T9"][0], zz["rho"][0], s["t_end"],
                          s["rtol"], s["atol"])
    top = gen.largest_species(tp["x"][-1:, :net.N], 2)[0]
    gY = np.zeros((2, 1, net.N))
    gY[0, 0, top[0]] = 1.0
    gY[1, 0, top[1]] = 1.0
    gE = np.zeros((2, 1)) if net.Q is not None else None
    dl, dY0, dT0, cnt, Yf, st = _gpu_adjoint(nb, torch, net, zz, s, gY, gE,
                                             np.zeros((2, 1)) if net.self_heating else None)
    assert st[0] == 0 and cnt[0, 0] == tp["counters"][0]
    rng = np.random.default_rng(4)
    eps = 1e-4
    for r in rng.choice(net.R, 3, replace=False):
        def run(sign):
            lm = np.zeros(net.R)
            lm[r] = sign * eps
            x, _ = oracle.replay(net, zz["Y"][0], zz["T9"][0], zz["rho"][0], tp["t"],
                                 tp["k"], s["rtol"], s["atol"], ln_mult=lm)
            return x
        fd = (run(1) - run(-1)) / (2 * eps)
        for q in range(2):
            y = abs(tp["x"][-1][top[q]])
            w = s["atol"] + s["rtol"] * y
            tol = 1e-6 * abs(fd[top[q]]) + 1e-3 * w / y * abs(fd[top[q]]) + 1e-13 * y
            assert abs(dl[q, 0, r] - fd[top[q]]) <= tol, (r, q, dl[q, 0, r], fd[top[q]])


def test_adjoint_cotangent_sets_are_independent_and_linear():
    nb, torch = nb_mod()
    net, z, s = gen.problem("chain13_heat", 64)
    rng = np.random.default_rng(2)
    g1 = rng.normal(size=(1, 64, net.N))
    g2 = rng.normal(size=(1, 64, net.N))
    e1, e2 = rng.normal(size=(1, 64)), rng.normal(size=(1, 64))
    t1, t2 = rng.normal(size=(1, 64)), rng.normal(size=(1, 64))
    both = _gpu_adjoint(nb, torch, net, z, s, np.concatenate([g1, g2]),
                        np.concatenate([e1, e2]), np.concatenate([t1, t2]))
    one = _gpu_adjoint(nb, torch, net, z, s, g1, e1, t1)
    two = _gpu_adjoint(nb, torch, net, z, s, g2, e2, t2)
    for k in range(3):
        assert np.array_equal(both[k][0], one[k][0])
        assert np.array_equal(both[k][1], two[k][0])
    summed = _gpu_adjoint(nb, torch, net, z, s, g1 + 2 * g2, e1 + 2 * e2, t1 + 2 * t2)
    for k in range(3):
        lin = one[k][0] + 2 * two[k][0]
        # linear up to rounding of the transposed solves
        np.testing.assert_allclose(summed[k][0], lin, rtol=1e-7,
                                   atol=1e-10 * np.abs(lin).max())


def test_autograd_function_gradients():
    nb, torch = nb_mod()
    net, z, s = gen.problem("net48_adjoint", 16)
    dev = torch.device("cuda")
    nc = nb.Network(net)
    Y0 = torch.from_numpy(z["Y"]).to(dev).requires_grad_(True)
    T9 = torch.from_numpy(z["T9"]).to(dev).requires_grad_(True)
    rho = torch.from_numpy(z["rho"]).to(dev)
    lm = torch.zeros(net.R, dtype=torch.float64, device=dev, requires_grad=True)
    Y, T9o, E, cnt, st = nb.Burn.apply(Y0, T9, rho, lm, nc, s["t_end"], s["rtol"], s["atol"])
    w = torch.from_numpy(np.random.default_rng(0).normal(size=(16, net.N))).to(dev)
    loss = (Y * w).sum() + 0.5 * E.sum()
    loss.backward()
    # same numbers from the explicit adjoint call
    dl, dY0, dT0, *_ = _gpu_adjoint(nb, torch, net, z, s, w.cpu().numpy()[None],
                                    np.full((1, 16), 0.5), None)
    np.testing.assert_allclose(lm.grad.cpu().numpy(), dl[0].sum(0), rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(Y0.grad.cpu().numpy(), dY0[0], rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(T9.grad.cpu().numpy(), dT0[0], rtol=1e-12, atol=1e-300)


def test_tape_capacity_is_reported():
    nb, torch = nb_mod()
    net, z, s = gen.problem("chain13_heat", 40)
    dl, dY0, dT0, cnt, _, st = _gpu_adjoint(nb, torch, net, z, s, np.ones((1, 40, net.N)),
                                            None, None, max_steps=50)
    full = st == 4
    assert full.any() and (cnt[full, 0] >= 50).all()
    assert (dl[0][full] == 0).all()
