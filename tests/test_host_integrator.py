"""The library's integrator source (the generic network and the shared BDF/
Newton code) compiled for the host and run zone by zone against the oracle,
for every rate form: fitted, effective (alpha,p)(p,gamma), screened and
tabulated.  A CPU check of the device code's integrator logic; the GPU tests
check the kernels themselves."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import gen
import oracle
from paper_2312_02836_gb300 import _topology, build
from tests.parity import compare

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def host_lib(tmp_path_factory):
    nvcc = shutil.which(os.environ.get("NVCC", "nvcc"))
    if nvcc is None:
        pytest.skip("no nvcc")
    build.build()          # writes the embedded-header file the sources include
    out = str(tmp_path_factory.mktemp("host") / "libhostint.so")
    csrc = os.path.join(ROOT, "paper_2312_02836_gb300", "csrc")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC",
                           "-Xcompiler", "-ffp-contract=off", "-shared",
                           "-I", os.path.join(ROOT, "include"), "-I", build.BUILD,
                           os.path.join(HERE, "host", "host_integrator.cu"),
                           os.path.join(csrc, "netload.cpp"), "-o", out],
                          stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
    lib = C.CDLL(out)
    V, D = C.c_void_p, C.c_double
    lib.host_burn.argtypes = [V, V, C.c_longlong, V, V, V, V, D, D, D, V, V, V, V, V]
    lib.host_burn.restype = C.c_int
    return lib


@pytest.mark.parametrize("name,Z", [("chain13_heat", 96), ("chain13_literal", 64),
                                    ("chain13_heat_ap", 96), ("chain13_heat_scr", 96),
                                    ("chain13_heat_tab", 96), ("net48", 24)])
def test_host_integrator_matches_oracle(host_lib, name, Z):
    net, z, s = gen.problem(name, Z)
    arrays, topo, coef = _topology(net)
    p = lambda a: None if a is None else a.ctypes.data
    Y = np.empty((Z, net.N)); T9 = np.empty(Z); E = np.empty(Z)
    cnt = np.zeros((Z, 9), np.int32); st = np.zeros(Z, np.int32)
    zeta = z.get("zeta")
    rc = host_lib.host_burn(C.byref(topo), coef, Z, p(z["Y"]), p(z["T9"]), p(z["rho"]),
                            p(zeta), s["t_end"], s["rtol"], s["atol"],
                            p(Y), p(T9), p(E), p(cnt), p(st))
    assert rc == 0
    run = lambda v: oracle.burn(net, z["Y"], z["T9"], z["rho"], s["t_end"], s["rtol"],
                                s["atol"], zeta=zeta, variant=v)
    o = run(0)
    rep = compare(dict(Y=Y, T9=T9, E=E, counters=cnt, status=st), o, s["atol"],
                  rtol=s["rtol"], variants=[run(v) for v in oracle.VARIANTS])
    assert (st == 0).all()
    print(name, rep)
