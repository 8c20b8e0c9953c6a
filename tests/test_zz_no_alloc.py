"""The allocation-free burn entry point, called through the C ABI.

It exists for callers that may not allocate device memory at burn time (a
solver whose device memory is reserved up front by its own pool, or code
that must not take the implicit synchronisation of cudaMalloc/cudaFree); it
keeps its scratch in an array compiled into the library.  It must give the
bits of the regular entry point on the generic kernel, call after call: the
shared scratch keeps the previous call's contents, so a second call checks
that nothing stale leaks in.  This file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


def _setup():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2312_02836_gb300 as nb
    from paper_2312_02836_gb300 import _abi
    return torch, nb, _abi, _abi.load()


def _noalloc(torch, abi, lib, nc, Z, Y0, T9, rho, s, t_end_zone=None, zeta=None,
             threads_per_block=0):
    dev = Y0.device
    opt = abi.Options()
    lib.nb_default_options(C.byref(opt))
    opt.threads_per_block = threads_per_block
    if t_end_zone is not None:
        opt.t_end_zone = t_end_zone.data_ptr()
    if zeta is not None:
        opt.zeta_zone = zeta.data_ptr()
    Y = torch.full_like(Y0, np.nan)
    T = torch.full_like(T9, np.nan)
    E = torch.full_like(T9, np.nan)
    cnt = torch.full((Z, abi.NCOUNT), -1, dtype=torch.int32, device=dev)
    st = torch.full((Z,), -1, dtype=torch.int32, device=dev)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.nb_burn_batch_noalloc(
        nc.handle, Z, Y0.data_ptr(), T9.data_ptr(), rho.data_ptr(),
        0.0 if t_end_zone is not None else s["t_end"], s["rtol"], s["atol"], None, 0,
        Y.data_ptr(), T.data_ptr(), E.data_ptr(), cnt.data_ptr(), st.data_ptr(),
        C.byref(opt), stream)
    assert rc == 0, lib.nb_strerror(rc)
    torch.cuda.synchronize()
    return dict(Y=Y.cpu().numpy(), T9=T.cpu().numpy(), E=E.cpu().numpy(),
                counters=cnt.cpu().numpy(), status=st.cpu().numpy())


# (workload, zones, per-zone end times): the self-heating chain; its
# screened form (per-zone plasma parameters); operator-split end times; and
# the 48-species network with enough zones that its 26 KB per-zone
# workspace caps the zones in flight to what fits the scratch array (about
# 1270 lanes), so lanes claim zones many times over
CASES = [("chain13_heat", 3000, False), ("chain13_heat_scr", 1500, False),
         ("chain13_heat", 1500, True), ("net48", 2500, False)]


@pytest.mark.parametrize("name,Z,split", CASES)
def test_noalloc_matches_regular_entry_point_twice(name, Z, split):
    torch, nb, abi, lib = _setup()
    dev = torch.device("cuda")
    net, z, s = gen.problem(name, Z)
    nc = nb.Network(net)
    Y0 = torch.from_numpy(z["Y"]).to(dev)
    T9 = torch.from_numpy(z["T9"]).to(dev)
    rho = torch.from_numpy(z["rho"]).to(dev)
    zeta = torch.from_numpy(z["zeta"]).to(dev) if "zeta" in z else None
    tz = None
    if split:
        tz = torch.from_numpy(np.exp(np.random.default_rng(5).uniform(
            np.log(1e-6), np.log(s["t_end"]), Z))).to(dev)
    if name == "net48":
        info = nc.info()
        lanes_fit = (32 << 20) // (8 * info["lane_doubles"])
        assert lanes_fit < Z and lanes_fit // 128 < torch.cuda.get_device_properties(
            dev).multi_processor_count
    ref = nb.burn(nc, Y0, T9, rho, s["t_end"] if tz is None else tz, s["rtol"], s["atol"],
                  specialize="generic", zeta=zeta)
    torch.cuda.synchronize()
    ref = {k: getattr(ref, k).cpu().numpy() for k in ("Y", "T9", "E", "counters", "status")}
    if zeta is not None:
        # the plasma parameter must matter, or the case checks nothing
        plain = nb.burn(nc, Y0, T9, rho, s["t_end"], s["rtol"], s["atol"], specialize="generic")
        assert not np.array_equal(plain.Y.cpu().numpy(), ref["Y"])
    for call in range(2):
        got = _noalloc(torch, abi, lib, nc, Z, Y0, T9, rho, s, tz, zeta)
        for k in ref:
            assert np.array_equal(got[k], ref[k]), (name, call, k)
    assert (ref["status"] == 0).all()


def test_noalloc_rejects_bad_arguments_and_oversized_networks():
    torch, nb, abi, lib = _setup()
    assert lib.nb_burn_batch_noalloc(None, 4, None, None, None, 1e-3, 1e-8, 1e-12, None, 0,
                                     None, None, None, None, None, None, None) == -1
    # 80 species, every one converting into every other: 6320 one-body rates
    # and a dense Jacobian, about 45,000 doubles of workspace per zone, so one
    # block of 128 zones needs more than the 32 MiB array
    N = 80
    pairs = [(i, j) for i in range(N) for j in range(N) if i != j]
    R = len(pairs)
    reac = np.full((R, 3), -1, np.int16)
    prod = np.full((R, 3), -1, np.int16)
    reac[:, 0] = [p[0] for p in pairs]
    prod[:, 0] = [p[1] for p in pairs]
    coeffs = np.zeros((R, 7))
    coeffs[:, 0] = -5.0
    spec = gen.NetworkSpec(name="dense80", N=N, R=R, reactants=reac, products=prod,
                           A=np.ones(N), coeffs=coeffs)
    nc = nb.Network(spec)
    assert nc.info()["lane_doubles"] * 8 * 128 > (32 << 20)
    dev = torch.device("cuda")
    Z = 4
    Y0 = torch.full((Z, N), 1.0 / N, dtype=torch.float64, device=dev)
    T9 = torch.ones(Z, dtype=torch.float64, device=dev)
    rho = torch.ones(Z, dtype=torch.float64, device=dev)
    out = torch.empty_like(Y0)
    T = torch.empty_like(T9)
    st = torch.empty(Z, dtype=torch.int32, device=dev)
    rc = lib.nb_burn_batch_noalloc(nc.handle, Z, Y0.data_ptr(), T9.data_ptr(), rho.data_ptr(),
                                   1.0, 1e-8, 1e-12, None, 0, out.data_ptr(), T.data_ptr(),
                                   None, None, st.data_ptr(), None, None)
    assert rc == -3, lib.nb_strerror(rc)
    # threads_per_block beyond 128 is refused
    opt = abi.Options()
    lib.nb_default_options(C.byref(opt))
    opt.threads_per_block = 256
    rc = lib.nb_burn_batch_noalloc(nc.handle, Z, Y0.data_ptr(), T9.data_ptr(), rho.data_ptr(),
                                   1.0, 1e-8, 1e-12, None, 0, out.data_ptr(), T.data_ptr(),
                                   None, None, st.data_ptr(), C.byref(opt), None)
    assert rc == -1
