"""ctypes front end of the plain FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke``
and by ``bench.py``'s CPU-baseline leg.  The library under
``paper_2312_02836_gb300`` never imports it, and it never imports the
library.  Inputs come from the seeded generators in ``gen``.

Every function restates the method of arXiv:2312.02836 Sec. 2-3 (generated
network RHS + analytic Jacobian, integrated per zone by a stiff BDF/Newton
integrator with optional self-heating); the C file's header lists the
integrator rules.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

N_COUNTERS = 9
COUNTER_NAMES = ("accepted", "rejected_error", "rejected_newton", "newton_iters",
                 "jacobians", "rhs_evals", "rate_evals", "edot_evals", "order_sum")
STATUS = {0: "OK", 1: "MAX_STEPS", 2: "DT_UNDERFLOW", 3: "NEWTON_FAIL",
          5: "NONFINITE", 7: "SINGULAR"}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off",
                           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm",
                           "-lpthread"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Net(C.Structure):
    _fields_ = [("N", C.c_int32), ("R", C.c_int32), ("self_heating", C.c_int32),
                ("reactants", C.c_void_p), ("products", C.c_void_p),
                ("Q", C.c_void_p), ("scale", C.c_void_p), ("coeffs", C.c_void_p),
                ("ap_pg", C.c_void_p), ("ap_coeffs", C.c_void_p),
                ("screen", C.c_void_p), ("tab_of", C.c_void_p),
                ("tab_nd", C.c_int32), ("tab_nt", C.c_int32),
                ("tab_dens", C.c_void_p), ("tab_t9", C.c_void_p),
                ("tab_lnl", C.c_void_p), ("charge", C.c_void_p)]


class _Opt(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("t_end", C.c_double),
                ("max_attempts", C.c_int32), ("newton_tol", C.c_double),
                ("newton_maxit", C.c_int32), ("fixed_h", C.c_double),
                ("fixed_order", C.c_int32), ("max_order", C.c_int32),
                ("variant", C.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
            lib.ora_rate_factors.argtypes = [P, D, D, D, D, P, P, P]
            lib.ora_rhs.argtypes = [P, P, D, D, D, D, P, P, P]
            lib.ora_jacobian.argtypes = [P, P, D, D, D, D, P, P]
            lib.ora_bdf_alpha.argtypes = [I32, D, P, D, P]
            lib.ora_extrapolate.argtypes = [I32, I32, P, P, D, P]
            lib.ora_burn_batch.argtypes = [P, P, I64, P, P, P, P, I32, P, P, P,
                                           P, P, I32, P, P]
            lib.ora_burn_batch.restype = I32
            lib.ora_burn_tape.argtypes = [P, P, P, D, D, D, P, P, P, P, P, I32, P,
                                          P, P, P, P, P]
            lib.ora_burn_tape.restype = I32
            lib.ora_replay.argtypes = [P, P, P, D, D, D, P, I32, P, P, D, I32, P, P]
            lib.ora_replay.restype = I32
            lib.ora_forward_sensitivity.argtypes = [P, D, D, D, P, I32, P, P, P, P, I32, P, P]
            lib.ora_forward_sensitivity.restype = I32
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class Network:
    """Oracle view of a network (anything with N, R, reactants, products,
    coeffs, Q, scale, self_heating attributes)."""

    def __init__(self, spec):
        self.N = int(spec.N)
        self.R = int(spec.R)
        self.self_heating = bool(spec.self_heating)
        self.reactants = np.ascontiguousarray(spec.reactants, dtype=np.int16)
        self.products = np.ascontiguousarray(spec.products, dtype=np.int16)
        self.coeffs = _f64(spec.coeffs)
        self.Q = _f64(getattr(spec, "Q", None))
        self.scale = _f64(getattr(spec, "scale", None))
        ap = getattr(spec, "ap_pg", None)
        self.ap_pg = None if ap is None else np.ascontiguousarray(ap, dtype=np.int8)
        self.ap_coeffs = _f64(getattr(spec, "ap_coeffs", None))
        self.screen = _f64(getattr(spec, "screen", None))
        tab = getattr(spec, "tab_of", None)
        self.tab_of = None if tab is None else np.ascontiguousarray(tab, dtype=np.int32)
        self.tab_dens = _f64(getattr(spec, "tab_dens", None))
        self.tab_t9 = _f64(getattr(spec, "tab_t9", None))
        self.tab_lnl = _f64(getattr(spec, "tab_lnl", None))
        self.charge = _f64(getattr(spec, "charge", None))
        if self.tab_of is not None:
            if self.tab_lnl is None or self.charge is None:
                raise ValueError("tab_of needs tab_dens, tab_t9, tab_lnl and charge")
            if self.ap_pg is not None and ((self.tab_of >= 0) & (self.ap_pg != 0)).any():
                raise ValueError("a reaction is either tabulated or effective")
        if self.ap_pg is not None and (self.ap_coeffs is None
                                       or self.ap_coeffs.size != 21 * self.R):
            raise ValueError("ap_pg needs ap_coeffs [R, 3, 7]")
        if self.self_heating and self.Q is None:
            raise ValueError("self-heating needs Q")
        self.n = self.N + (1 if self.self_heating else 0)
        self._s = _Net(self.N, self.R, int(self.self_heating),
                       _p(self.reactants), _p(self.products), _p(self.Q),
                       _p(self.scale), _p(self.coeffs), _p(self.ap_pg),
                       _p(self.ap_coeffs), _p(self.screen), _p(self.tab_of),
                       0 if self.tab_dens is None else self.tab_dens.size,
                       0 if self.tab_t9 is None else self.tab_t9.size,
                       _p(self.tab_dens), _p(self.tab_t9), _p(self.tab_lnl),
                       _p(self.charge))

    @property
    def ptr(self):
        return C.addressof(self._s)


def _net(net):
    return net if isinstance(net, Network) else Network(net)


# rounding variants of the oracle (bits of ``variant``): equally valid
# orderings of the same arithmetic, used to measure how far rounding alone
# moves a burn.  SUM_REVERSE: sums in decreasing index order; LU_REVERSE: the
# index-reversed Newton matrix is factored; ULP: exp, log and cbrt one ulp
# off; STEP_EXP: the step-size factor through exp and log instead of pow;
# LU_PERMUTE: the Newton matrix factored in a fixed pseudo-random index order.
VARIANT_SUM_REVERSE, VARIANT_LU_REVERSE, VARIANT_ULP, VARIANT_STEP_EXP = 1, 2, 4, 8
VARIANT_LU_PERMUTE = 16
# the set a parity check measures the oracle's own spread with: each
# variant alone and all of them at once
VARIANTS = (VARIANT_SUM_REVERSE, VARIANT_LU_REVERSE, VARIANT_ULP, VARIANT_STEP_EXP,
            VARIANT_LU_PERMUTE, 31)


def _opts(t_end, rtol, atol, max_attempts=500000, newton_tol=1e-3,
          newton_maxit=4, fixed_h=0.0, fixed_order=0, max_order=5, variant=0):
    return _Opt(rtol, atol, t_end, max_attempts, newton_tol, newton_maxit,
                fixed_h, fixed_order, max_order, variant)


def rate_factors(net, T9, rho, ln_mult=None, zeta=0.0, ye=1.0):
    """k_r = s_r e^p_r rho^(n_r-1) lambda_r(T9) exp(H_r) and d ln k_r / dT9
    (H_r the weak-screening exponent at plasma parameter zeta; tabulated
    rates read at log10(rho ye))."""
    net = _net(net)
    lib = _load()
    k = np.empty(net.R)
    g = np.empty(net.R)
    lm = _f64(ln_mult)
    lib.ora_rate_factors(net.ptr, float(T9), float(rho), float(zeta), float(ye), _p(lm),
                         _p(k), _p(g))
    return k, g


def rhs(net, x, T9=0.0, rho=1.0, ln_mult=None, zeta=0.0, ye=1.0):
    """f(x) [n] and edot at state x (x[N] is T9 under self-heating)."""
    net = _net(net)
    lib = _load()
    x = _f64(x)
    f = np.empty(net.n)
    ed = C.c_double(0.0)
    lm = _f64(ln_mult)
    lib.ora_rhs(net.ptr, _p(x), float(T9), float(rho), float(zeta), float(ye), _p(lm), _p(f),
                C.byref(ed))
    return f, ed.value


def jacobian(net, x, T9=0.0, rho=1.0, ln_mult=None, zeta=0.0, ye=1.0):
    """Analytic Jacobian df/dx [n, n]."""
    net = _net(net)
    lib = _load()
    x = _f64(x)
    J = np.empty((net.n, net.n))
    lm = _f64(ln_mult)
    lib.ora_jacobian(net.ptr, _p(x), float(T9), float(rho), float(zeta), float(ye), _p(lm),
                     _p(J))
    return J


def bdf_alpha(k, t_new, t_old, h):
    """alpha_0..alpha_k of the variable-step BDF formula of order k."""
    lib = _load()
    t_old = _f64(np.asarray(t_old, dtype=np.float64))
    a = np.empty(k + 1)
    lib.ora_bdf_alpha(int(k), float(t_new), _p(t_old), float(h), _p(a))
    return a


def extrapolate(t_pts, x_pts, t):
    """Value at t of the polynomial through (t_pts[j], x_pts[j])."""
    lib = _load()
    t_pts = _f64(np.asarray(t_pts, dtype=np.float64))
    x_pts = _f64(np.atleast_2d(np.asarray(x_pts, dtype=np.float64)))
    q = t_pts.shape[0] - 1
    n = x_pts.shape[1]
    out = np.empty(n)
    lib.ora_extrapolate(q, n, _p(t_pts), _p(x_pts), float(t), _p(out))
    return out


def burn(net, Y0, T9, rho, t_end, rtol, atol, ln_mult=None, threads=0, zeta=None,
         **opts):
    """Burn Z zones.  t_end is a number or a per-zone array [Z]; zeta None or
    the per-zone plasma parameters [Z] for screening.  Returns
    dict(Y, T9, E, counters [Z, 9], status, threads)."""
    net = _net(net)
    lib = _load()
    Y0 = _f64(np.atleast_2d(Y0))
    Z = Y0.shape[0]
    T9 = _f64(np.broadcast_to(np.asarray(T9, dtype=np.float64), (Z,)))
    rho = _f64(np.broadcast_to(np.asarray(rho, dtype=np.float64), (Z,)))
    per_zone = 0
    lm = None
    if ln_mult is not None:
        lm = _f64(ln_mult)
        per_zone = 1 if lm.ndim == 2 else 0
    Y = np.empty((Z, net.N))
    T9o = np.empty(Z)
    E = np.empty(Z)
    cnt = np.zeros((Z, N_COUNTERS), dtype=np.int32)
    st = np.zeros(Z, dtype=np.int32)
    tz = None
    if np.ndim(t_end) > 0:
        tz = _f64(t_end)
        t_end = 0.0
    zt = None if zeta is None else _f64(np.broadcast_to(np.asarray(zeta, dtype=np.float64), (Z,)))
    o = _opts(float(t_end), rtol, atol, **opts)
    used = lib.ora_burn_batch(net.ptr, C.addressof(o), Z, _p(Y0), _p(T9),
                              _p(rho), _p(lm), per_zone, _p(Y), _p(T9o), _p(E),
                              _p(cnt), _p(st), int(threads), _p(tz), _p(zt))
    return dict(Y=Y, T9=T9o, E=E, counters=cnt, status=st, threads=used)


def burn_tape(net, Y0, T9, rho, t_end, rtol, atol, ln_mult=None, cap=200000,
              zeta=0.0, **opts):
    """One zone with its accepted schedule: dict(Y, T9, E, counters, status,
    t [S+1], k [S+1], x [S+1, n], Ehist [S+1], hnext [S+1]); hnext[s] is the
    step size the controller chose after accepted step s."""
    net = _net(net)
    lib = _load()
    Y0 = _f64(Y0)
    lm = _f64(ln_mult)
    Y = np.empty(net.N)
    T9o = C.c_double(0.0)
    E = C.c_double(0.0)
    cnt = np.zeros(N_COUNTERS, dtype=np.int32)
    tt = np.empty(cap)
    tk = np.empty(cap, dtype=np.int32)
    tx = np.empty((cap, net.n))
    tE = np.empty(cap)
    th = np.full(cap, np.nan)
    count = C.c_int32(0)
    o = _opts(t_end, rtol, atol, **opts)
    st = lib.ora_burn_tape(net.ptr, C.addressof(o), _p(Y0), float(T9),
                           float(rho), float(zeta), _p(lm), _p(Y), C.byref(T9o), C.byref(E),
                           _p(cnt), cap, _p(tt), _p(tk), _p(tx), _p(tE),
                           C.byref(count), _p(th))
    c = count.value
    return dict(Y=Y, T9=T9o.value, E=E.value, counters=cnt, status=st,
                t=tt[:c].copy(), k=tk[:c].copy(), x=tx[:c].copy(),
                Ehist=tE[:c].copy(), hnext=th[:c].copy())


def replay(net, Y0, T9, rho, t, k, rtol, atol, ln_mult=None, tol=1e-6,
           maxit=50, zeta=0.0):
    """Final (x [n], E) of the frozen schedule (t, k), full Newton to tol
    (weighted norm) and one further iteration."""
    net = _net(net)
    lib = _load()
    Y0 = _f64(Y0)
    lm = _f64(ln_mult)
    t = _f64(t)
    k = np.ascontiguousarray(k, dtype=np.int32)
    x = np.empty(net.n)
    E = C.c_double(0.0)
    o = _opts(float(t[-1]), rtol, atol)
    rc = lib.ora_replay(net.ptr, C.addressof(o), _p(Y0), float(T9), float(rho),
                        float(zeta), _p(lm), int(t.shape[0] - 1), _p(t), _p(k), float(tol),
                        int(maxit), _p(x), C.byref(E))
    if rc != 0:
        raise RuntimeError("replay did not converge")
    return x, E.value


def forward_sensitivity(net, T9, rho, t, k, x, ln_mult=None, zeta=0.0, h=None, variant=0):
    """d x_final / d theta [n, P] and d E_final / d theta [P] along a recorded
    schedule; theta = (ln multipliers [R], x0 [n], T9 if not self-heating).
    h: the step sizes of the record (default t_s - t_{s-1}); variant: the
    rounding variant bits (see VARIANTS)."""
    net = _net(net)
    lib = _load()
    lm = _f64(ln_mult)
    t = _f64(t)
    k = np.ascontiguousarray(k, dtype=np.int32)
    x = _f64(x)
    h = _f64(h)
    P = net.R + net.n + (0 if net.self_heating else 1)
    dx = np.empty((net.n, P))
    dE = np.empty(P)
    rc = lib.ora_forward_sensitivity(net.ptr, float(T9), float(rho), float(zeta), _p(lm),
                                     int(t.shape[0] - 1), _p(t), _p(k), _p(x), _p(h),
                                     int(variant), _p(dx), _p(dE))
    if rc != 0:
        raise RuntimeError("singular Newton matrix in forward sensitivity")
    return dx, dE
