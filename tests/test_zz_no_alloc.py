"""The allocation-free burn entry point, called through the C ABI.

It exists for callers that may not allocate device memory at burn time; it
keeps its scratch in an array compiled into the library.  It must give the
results of the regular entry point, call after call (the shared scratch keeps
the previous call's contents, so a second call checks that nothing stale
leaks in).  This file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_entry_point_twice():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2312_02836_gb300 as nb
    from paper_2312_02836_gb300 import _abi

    lib = _abi.load()
    dev = torch.device("cuda")
    for name, Z in (("chain13_heat", 3000), ("net48", 96)):
        net, z, s = gen.problem(name, Z)
        nc = nb.Network(net)
        Y0 = torch.from_numpy(z["Y"]).to(dev)
        T9 = torch.from_numpy(z["T9"]).to(dev)
        rho = torch.from_numpy(z["rho"]).to(dev)
        ref = nb.burn(nc, Y0, T9, rho, s["t_end"], s["rtol"], s["atol"])
        torch.cuda.synchronize()
        opt = _abi.Options()
        lib.nb_default_options(C.byref(opt))
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        for call in range(2):
            Y = torch.full_like(Y0, np.nan)
            T = torch.full_like(T9, np.nan)
            E = torch.full_like(T9, np.nan)
            cnt = torch.full((Z, 8), -1, dtype=torch.int32, device=dev)
            st = torch.full((Z,), -1, dtype=torch.int32, device=dev)
            rc = lib.nb_burn_batch_noalloc(
                nc.handle, Z, Y0.data_ptr(), T9.data_ptr(), rho.data_ptr(),
                s["t_end"], s["rtol"], s["atol"], None, 0, Y.data_ptr(), T.data_ptr(),
                E.data_ptr(), cnt.data_ptr(), st.data_ptr(), C.byref(opt), stream)
            assert rc == 0, lib.nb_strerror(rc)
            torch.cuda.synchronize()
            Yr, Yn = ref.Y.cpu().numpy(), Y.cpu().numpy()
            # the parity bar of the GPU tests: 1e-9 |Y| + 1e-5 atol
            assert np.all(np.abs(Yn - Yr) <= 1e-9 * np.abs(Yr) + 1e-5 * s["atol"]), (name, call)
            np.testing.assert_allclose(T.cpu().numpy(), ref.T9.cpu().numpy(), rtol=1e-9)
            np.testing.assert_allclose(E.cpu().numpy(), ref.E.cpu().numpy(), rtol=1e-9, atol=1e-12)
            assert np.array_equal(st.cpu().numpy(), ref.status.cpu().numpy())
            assert np.array_equal(cnt.cpu().numpy(), ref.counters.cpu().numpy())


def test_noalloc_rejects_bad_arguments():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2312_02836_gb300 import _abi
    lib = _abi.load()
    assert lib.nb_burn_batch_noalloc(None, 4, None, None, None, 1e-3, 1e-8, 1e-12, None, 0,
                                     None, None, None, None, None, None, None) == -1
