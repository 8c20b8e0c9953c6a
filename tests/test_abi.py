"""The C ABI library builds, loads and exports every symbol its header
declares; argument errors are caught on the host before any GPU work; the
Python package refuses to run without a GPU.  No compute call here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import gen
from paper_2312_02836_gb300 import _abi, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "netburn.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z0-9_]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    lib = C.CDLL(build.build())
    names = declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(_abi.EXPORTS)


def test_strerror_and_defaults_without_gpu():
    lib = _abi.load()
    assert lib.nb_strerror(0) == b"ok"
    assert b"topology" in lib.nb_strerror(-2)
    o = _abi.Options()
    lib.nb_default_options(C.byref(o))
    assert o.max_attempts == 500000 and o.kernel == 0 and o.blob_in_shared == -1


def _topo(net, reactants=None):
    reac = np.ascontiguousarray(net.reactants if reactants is None else reactants, np.int16)
    prod = np.ascontiguousarray(net.products, np.int16)
    t = _abi.Topology(net.N, net.R, reac.ctypes.data, prod.ctypes.data,
                      None, None, int(net.self_heating))
    return t, reac, prod


def test_bad_topology_rejected_on_host():
    lib = _abi.load()
    net = gen.network("chain13")
    bad = net.reactants.copy()
    bad[3, 1] = 13                       # species index out of range
    t, _r, _p = _topo(net, bad)
    h = C.c_void_p()
    coef = np.ascontiguousarray(net.coeffs)
    assert lib.nb_net_load(C.byref(t), coef.ctypes.data, C.byref(h)) == -2
    empty = net.reactants.copy()
    empty[0] = -1                        # reaction without reactants
    t, _r, _p = _topo(net, empty)
    assert lib.nb_net_load(C.byref(t), coef.ctypes.data, C.byref(h)) == -2
    # self-heating without Q, non-finite coefficient
    t, _r, _p = _topo(net)
    t.self_heating = 1
    assert lib.nb_net_load(C.byref(t), coef.ctypes.data, C.byref(h)) == -1
    t.self_heating = 0
    c2 = coef.copy()
    c2[2, 3] = np.nan
    assert lib.nb_net_load(C.byref(t), c2.ctypes.data, C.byref(h)) == -1
    assert lib.nb_net_load(None, coef.ctypes.data, C.byref(h)) == -1


def test_burn_argument_checks_on_host():
    lib = _abi.load()
    # a null network handle is rejected before any device work
    assert lib.nb_burn_batch(None, 4, None, None, None, 1.0, 1e-8, 1e-12, None, 0,
                             None, None, None, None, None, None, None, None) == -1
    assert lib.nb_tape_alloc(None, 4, 10, 0, None) == -1


def test_package_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2312_02836_gb300 as nb
    with pytest.raises(nb.NetburnError):
        nb.Network(gen.network("chain13"))


def test_multi_network_argument_checks_on_host():
    # set counts and tolerances are checked before any device work
    lib = _abi.load()
    sets = (_abi.BurnSet * 13)()
    assert lib.nb_burn_multi(0, sets, 1.0, 1e-8, 1e-12, None, None) == -1
    assert lib.nb_burn_multi(13, sets, 1.0, 1e-8, 1e-12, None, None) == -1
    assert lib.nb_burn_multi(1, None, 1.0, 1e-8, 1e-12, None, None) == -1
    assert lib.nb_burn_multi(1, sets, 1.0, -1e-8, 1e-12, None, None) == -1
    assert lib.nb_burn_multi(1, sets, float("nan"), 1e-8, 1e-12, None, None) == -1


def test_autotune_candidates_per_network():
    from paper_2312_02836_gb300.autotune import (COOP_CANDIDATES, GENERIC_CANDIDATES,
                                                 SPECIALIZED_CANDIDATES, eligible)
    # a large network with no generated kernel: generic lane and warp kernels
    big = eligible(dict(specialize_auto=False, n_state=48))
    assert big == list(GENERIC_CANDIDATES) + list(COOP_CANDIDATES)
    # a small network that has one: lane kernels only, generated ones included
    small = eligible(dict(specialize_auto=True, n_state=14))
    assert small == list(GENERIC_CANDIDATES) + list(SPECIALIZED_CANDIDATES)
