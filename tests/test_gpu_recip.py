"""The integrator's Newton-Raphson reciprocals on the GPU against the
correctly rounded 1/a (CUDA's division): recip2, used for the LU pivots, to
within 2 ulp; recip1, used for the error weights, to 2^-38 relative (the seed
instruction has about 20 good bits, measured 2^-39.9 after one step); both
exact on the inputs outside the normal range, which take the division."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _lib(tmp_path):
    from paper_2312_02836_gb300 import build
    nvcc = shutil.which(os.environ.get("NVCC", "nvcc"))
    assert nvcc, "nvcc needed"
    build.build()          # the embedded-header file the sources include
    out = str(tmp_path / "librecip.so")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                           "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "include"), "-I", build.BUILD,
                           os.path.join(HERE, "host", "recip_check.cu"), "-o", out])
    lib = C.CDLL(out)
    lib.recip_eval.argtypes = [C.c_void_p, C.c_longlong, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.recip_eval.restype = C.c_int
    return lib


def test_newton_raphson_reciprocals(tmp_path):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    lib = _lib(tmp_path)
    rng = np.random.default_rng(5)
    # the ranges the integrator meets (weights atol + rtol |x| from 1e-12 up,
    # pivots around alpha0 = O(1) and far from it), both signs, every
    # mantissa, and the edges of the normal range
    a = np.concatenate([
        rng.uniform(1.0, 2.0, 200000) * 2.0 ** rng.integers(-1000, 1000, 200000),
        -rng.uniform(1.0, 2.0, 50000) * 2.0 ** rng.integers(-60, 60, 50000),
        np.array([1.0, -1.0, 3.0, 2.0 ** -1021, 2.0 ** 1020, 1.5 * 2.0 ** 1021,
                  1.5 * 2.0 ** 1022, np.finfo(float).tiny, 5e-324, 0.0, -0.0, np.inf,
                  np.nan]),
    ])
    n = a.size
    r1, r2, rd = np.empty(n), np.empty(n), np.empty(n)
    assert lib.recip_eval(a.ctypes.data, n, r1.ctypes.data, r2.ctypes.data, rd.ctypes.data) == 0
    with np.errstate(divide="ignore", invalid="ignore"):
        exact = 1.0 / a
    np.testing.assert_array_equal(rd, exact)
    fin = np.isfinite(exact) & (exact != 0)
    ulp = np.spacing(np.abs(exact[fin]))
    e2 = np.abs(r2[fin] - exact[fin]) / ulp
    e1 = np.abs(r1[fin] - exact[fin]) / np.abs(exact[fin])
    print(f"recip2: max {e2.max():.2f} ulp, {np.mean(e2 > 0):.3%} not correctly rounded; "
          f"recip1: max relative error {e1.max():.3g} = 2^{np.log2(max(e1.max(), 1e-300)):.1f}")
    assert e2.max() <= 2.0
    assert e1.max() <= 2.0 ** -38
    # outside the normal range both take the division
    odd = ~fin | (np.abs(a) < 2.0 ** -1022) | (np.abs(a) >= 2.0 ** 1022)
    np.testing.assert_array_equal(r1[odd], exact[odd])
    np.testing.assert_array_equal(r2[odd], exact[odd])
