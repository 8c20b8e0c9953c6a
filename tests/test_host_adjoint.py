"""The library's forward burn with a tape and its checkpointed reverse sweep
(the generic network, adjoint.cuh) compiled for the host, against the
oracle's forward sensitivity along the same recorded trajectory, on the CPU.
Checks the recomputation of checkpointed blocks (every stride gives the
same bits) and the gradients (the bar of tests/sensitivity.py) without a
GPU; the GPU tests check the kernel itself."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import gen
import oracle
from paper_2312_02836_gb300 import _topology, build
from tests.sensitivity import check_zone, cotangents, oracle_sensitivities

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def host_lib(tmp_path_factory):
    nvcc = shutil.which(os.environ.get("NVCC", "nvcc"))
    if nvcc is None:
        pytest.skip("no nvcc")
    build.build()          # writes the embedded-header file the sources include
    out = str(tmp_path_factory.mktemp("hostadj") / "libhostadj.so")
    csrc = os.path.join(ROOT, "paper_2312_02836_gb300", "csrc")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC",
                           "-Xcompiler", "-ffp-contract=off", "-shared",
                           "-I", os.path.join(ROOT, "include"), "-I", build.BUILD,
                           os.path.join(HERE, "host", "host_adjoint.cu"),
                           os.path.join(csrc, "netload.cpp"), "-o", out],
                          stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
    lib = C.CDLL(out)
    V, D, I, L = C.c_void_p, C.c_double, C.c_int, C.c_longlong
    lib.host_adjoint.argtypes = [V, V, L, V, V, V, V, D, D, D, I, I, I, I, V, V, V] + [V] * 12
    lib.host_adjoint.restype = C.c_int
    return lib


def host_run(lib, net, z, s, stride, gY, gE, gT9, cap=6000):
    Z = z["T9"].shape[0]
    n = net.N + int(net.self_heating)
    K = gY.shape[0]
    arrays, topo, coef = _topology(net)
    scap = 1 + ((cap - 1 + stride - 1) // stride) * min(stride, 7)
    out = dict(Y=np.empty((Z, net.N)), T9=np.empty(Z), E=np.empty(Z),
               counters=np.zeros((Z, 9), np.int32), status=np.zeros(Z, np.int32),
               sched=np.zeros((Z, cap, 2)), ord=np.zeros((Z, cap), np.int8),
               states=np.full((Z, scap, n + 1), np.nan), steps=np.zeros(Z, np.int32),
               dl=np.zeros((K, Z, net.R)), dY0=np.zeros((K, Z, net.N)), dT0=np.zeros((K, Z)))
    p = lambda a: None if a is None else np.ascontiguousarray(a).ctypes.data
    keep = [np.ascontiguousarray(a) for a in (gY, gE, gT9) if a is not None]
    rc = lib.host_adjoint(C.byref(topo), coef, Z, p(z["Y"]), p(z["T9"]), p(z["rho"]),
                          p(z.get("zeta")), s["t_end"], s["rtol"], s["atol"], cap, stride, scap,
                          K, p(keep[0]), p(gE if gE is None else keep[1]),
                          p(None if gT9 is None else keep[-1]),
                          *(p(out[k]) for k in ("Y", "T9", "E", "counters", "status", "sched",
                                                "ord", "states", "steps", "dl", "dY0", "dT0")))
    assert rc == 0

    def read(i):
        S = out["steps"][i]
        slots = [0] + [1 + ((q - 1) // stride) * min(stride, 7) +
                       ((q - 1) % stride - (stride - min(stride, 7))) for q in range(1, S)]
        return dict(t=out["sched"][i, :S, 0], h=out["sched"][i, :S, 1],
                    k=out["ord"][i, :S].astype(np.int32),
                    x=out["states"][i, slots, :n] if stride == 1 else None)
    out["read"] = read
    return out


@pytest.mark.parametrize("name,Z", [("chain13_heat", 12), ("net48_adjoint", 4),
                                    ("chain13_heat_scr", 6), ("chain13_heat_ap", 6),
                                    ("chain13_heat_tab", 6)])
def test_host_adjoint_matches_oracle_sensitivity(host_lib, name, Z):
    net, z, s = gen.problem(name, Z)
    o = oracle.burn(net, z["Y"], z["T9"], z["rho"], s["t_end"], s["rtol"], s["atol"],
                    zeta=z.get("zeta"))
    gY, gE = cotangents(net, o["Y"], Z)
    gT9 = np.zeros((6, Z)) if net.self_heating else None
    full = host_run(host_lib, net, z, s, 1, gY, gE, gT9)
    assert (full["status"] == 0).all()
    for stride in (2, 7, 16):
        part = host_run(host_lib, net, z, s, stride, gY, gE, gT9)
        for k in ("dl", "dY0", "dT0", "Y"):
            assert np.array_equal(part[k], full[k]), (stride, k)
    sens = oracle_sensitivities(net, z, full["read"], range(Z))
    lit = tot = 0
    for i in range(Z):
        a, b = check_zone(net, gY, gE, gT9, full, sens, i)
        lit += a
        tot += b
    print(name, f"entries beyond 1e-10 relative (within the measured spread): {lit}/{tot}")
