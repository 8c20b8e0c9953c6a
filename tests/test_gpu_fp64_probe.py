"""The FP64 pipe rate of the GPU (the burn's roofline denominator), measured
with the DFMA microbenchmark in ``tests/host/fp64_probe.cu``, against the
peak derived from the unit counts: 152 SMs x 2 FP64 FMA lanes per clock x 2
flops x 2.07 GHz.  Run with ``-s`` to print the table of the profile
summary."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def probe_lib(tmp_path):
    nvcc = shutil.which(os.environ.get("NVCC", "nvcc"))
    assert nvcc, "nvcc needed"
    out = str(tmp_path / "libfp64probe.so")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                           "-Xcompiler", "-fPIC", "-shared",
                           os.path.join(HERE, "host", "fp64_probe.cu"), "-o", out])
    lib = C.CDLL(out)
    lib.fp64_probe.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]
    lib.fp64_probe.restype = C.c_int
    return lib


def test_fp64_rate_matches_derived_peak(tmp_path):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    from paper_2312_02836_gb300 import metrics
    lib = probe_lib(tmp_path)
    rates = {}
    for active in (32, 16, 8, 1):
        tf, ms = C.c_double(), C.c_double()
        assert lib.fp64_probe(active, 4096, 4, C.byref(tf), C.byref(ms)) == 0
        rates[active] = tf.value
        print(f"active lanes {active:2d}: {tf.value:.4f} TFLOP/s ({ms.value:.2f} ms)")
    assert 0.85 * metrics.FP64_PEAK_TFLOPS <= rates[32] <= 1.05 * metrics.FP64_PEAK_TFLOPS
    # an FP64 warp instruction costs the pipe the same whatever its active
    # lanes: the useful rate scales with them
    assert rates[8] < 0.35 * rates[32]
