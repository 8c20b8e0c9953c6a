"""The network-specialised kernel's generator and its run-time compilation,
on the CPU (the CUDA run-time compiler needs no GPU).  Its results are
checked against the generic kernel, bit for bit, by the GPU tests."""
import ctypes as C
import re

import numpy as np
import pytest

import gen
import paper_2312_02836_gb300 as nb
from paper_2312_02836_gb300 import _abi


def test_source_spells_out_the_network():
    net = gen.network("chain13_heat")
    src = nb.specialized_source(net, 0)
    head = src.splitlines()[0]
    assert "N = 13 species, R = 12 reactions, n = 14" in head
    assert "storage variant 2" in head        # 7n + LU slots > 160: LU in memory
    # one exponent, one rate and one derivative factor per reaction, with the
    # fit coefficients as exact hexadecimal literals
    assert len(re.findall(r"^  e = rate_exponent\(", src, re.M)) == net.R
    # the rates near the attempt's reference temperature: one small-delta
    # update per reaction, with the full exponent as its fallback
    assert len(re.findall(r"rate_near\(w\.kp\[\d+\], de\)", src)) == net.R
    assert len(re.findall(r"^      e = rate_exponent\(", src, re.M)) == net.R
    assert src.count("else full |= 1ull << ") == net.R     # fallbacks grouped apart
    assert len(re.findall(r"^  w\.k\[\d+\] = exp_tang\(e\)", src, re.M)) == net.R
    assert len(re.findall(r"^      w\.k\[\d+\] = exp_tang\(e\)", src, re.M)) == net.R
    assert len(re.findall(r"w\.g\[\d+\] = rate_dlog\(", src)) == net.R
    a = net.coeffs[5]
    assert float.hex(float(a[0])).replace("0x", "") in src.replace("0x", "")
    # every reaction's term multiplies its reactants: 3 Y0 for the 3-alpha
    # reaction, Y_i Y0 for the captures
    assert "w.rr[0] = w.k[0] * v[0] * v[0] * v[0];" in src
    assert "w.rr[1] = w.k[1] * v[0] * v[1];" in src or "w.rr[1] = w.k[1] * v[1] * v[0];" in src
    assert "extern \"C\" __global__" in src and "nb_spec_burn" in src
    # variants differ only in where work arrays live
    assert "double lu[" in nb.specialized_source(net, 1)
    assert "LV lu;" in nb.specialized_source(net, 2)
    assert "LV psi, iw, xp, tmp;" in nb.specialized_source(net, 3)
    # fixed temperature: no derivative factors, rates kept for the whole zone
    src0 = nb.specialized_source(gen.network("chain13"), 1)
    assert "rate_dlog" not in src0 and "LV k;" in src0


def test_source_arguments_checked():
    lib = _abi.load()
    net = gen.network("chain13")
    arrays, topo, coef = nb._topology(net)
    n = C.c_int64()
    assert lib.nb_specialize_source(None, coef, 0, None, 0, None) == -1
    assert lib.nb_specialize_source(C.byref(topo), coef, 4, None, 0,
                                    C.byref(n)) == -1
    # a too-small buffer reports the needed length and fails
    rc = lib.nb_specialize_source(C.byref(topo), coef, 0, None, 0,
                                  C.byref(n))
    assert rc == -1 and n.value > 1000


@pytest.mark.parametrize("name", ["chain13_heat", "chain13", "chain13_heat_ap",
                                  "chain13_heat_scr", "chain13_heat_tab"])
def test_specialized_kernel_compiles_for_sm103a(name):
    try:
        log = nb.specialize_compile(gen.network(name), 0)
    except nb.NetburnError as e:
        if "libnvrtc not found" in str(e):
            pytest.skip("no run-time compiler in this image")
        raise
    assert "nb_spec_burn" in log and "sm_103a" in log
    m = re.search(r"Used (\d+) registers", log)
    assert m and int(m.group(1)) <= 255


def test_effective_rates_in_the_source_and_checked_on_load():
    # every (alpha,p)(p,gamma) rate combines its four channels through the
    # shared helper, in the full evaluation and as the near evaluation's only
    # path
    net = gen.network("chain13_heat_ap")
    n_ap = int(net.ap_pg.sum())
    src = nb.specialized_source(net, 0)
    assert src.count("const APRate q = ap_rate(e, eap, epg, epa);") == 2 * n_ap
    assert src.count("w.g[") >= n_ap and "ap_dlog(q," in src
    # a flag other than 0/1, a non-finite channel fit: rejected on the host
    lib = _abi.load()
    n = C.c_int64()
    for bad in ("flag", "fit"):
        spec = gen.network("chain13_heat_ap")
        if bad == "flag":
            spec.ap_pg = spec.ap_pg.copy()
            spec.ap_pg[3] = 2
        else:
            spec.ap_coeffs = spec.ap_coeffs.copy()
            spec.ap_coeffs[4, 1, 2] = float("nan")
        arrays, topo, coef = nb._topology(spec)
        assert lib.nb_specialize_source(C.byref(topo), coef, 0, None, 0, C.byref(n)) == -1


def test_screening_in_the_source():
    # a screened network adds s_r * hz to every exponent (full and near
    # evaluations) and s_r * hzd to every d ln k / dT9
    net = gen.network("chain13_heat_scr")
    src = nb.specialized_source(net, 0)
    assert src.count(", p.hz, e);") == 2 * net.R      # full, and near's fallback
    assert src.count(", d.d7, de);") == net.R
    assert src.count(", p.hzd, rate_dlog(") == net.R
    assert "p.hz" not in nb.specialized_source(gen.network("chain13_heat"), 0)
    # a negative strength is rejected on the host
    spec = gen.network("chain13_heat_scr")
    spec.screen = spec.screen.copy()
    spec.screen[2] = -1.0
    arrays, topo, coef = nb._topology(spec)
    n = C.c_int64()
    assert _abi.load().nb_specialize_source(C.byref(topo), coef, 0, None, 0,
                                            C.byref(n)) == -1


def test_tables_in_the_source():
    # the tables are literal device arrays; every tabulated rate reads its
    # table in the full evaluation and takes it (not the near update) in the
    # near evaluation; the zone's Ye comes from the literal charges
    net = gen.network("chain13_heat_tab")
    n_tab = int((net.tab_of >= 0).sum())
    src = nb.specialized_source(net, 0)
    assert "__device__ const double NB_TAB_L[%d]" % net.tab_lnl.size in src
    assert src.count("e = table_lnl(NB_TAB_L + ") == 2 * n_tab
    assert src.count("rate_near(w.kp[") == net.R - n_tab
    assert src.count("ye = fma(") == net.N
    # tabulated and effective at once: rejected on the host
    spec = gen.network("chain13_heat_tab")
    spec.ap_pg = np.zeros(spec.R, dtype=np.int8)
    spec.ap_pg[2] = 1
    spec.ap_coeffs = np.zeros((spec.R, 3, 7))
    arrays, topo, coef = nb._topology(spec)
    n = C.c_int64()
    assert _abi.load().nb_specialize_source(C.byref(topo), coef, 0, None, 0,
                                            C.byref(n)) == -1
