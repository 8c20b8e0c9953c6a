"""GB300 batched stiff reaction-network burner (arXiv:2312.02836).

Python binding of the C ABI in ``include/netburn.h``.  PyTorch supplies the
device memory and the stream; every step of the burn runs in the CUDA
library (``_build/libnetburn.so``).  There is no CPU path: without a CUDA
device the calls raise.

    net = Network(spec)                       # compile a network
    out = burn(net, Y0, T9, rho, t_end, rtol, atol)   # torch CUDA float64
    Y, T9, E, counters, status = Burn.apply(Y0, T9, rho, ln_mult, net, t_end, rtol, atol)
"""
from __future__ import annotations

import ctypes as C
from typing import NamedTuple, Optional

import numpy as np

from . import _abi
from ._abi import (COUNTER_NAMES, KERNEL_COOP, KERNEL_PERSISTENT, KERNEL_PLAIN, NCOUNT,
                   ZONE_STATUS, NetburnError)

__all__ = ["Network", "specialized_source", "specialize_compile", "burn", "burn_multi", "burn_host", "BurnGraph", "Tape", "adjoint", "Burn", "zone_costs",
           "BurnResult", "NetburnError", "COUNTER_NAMES", "ZONE_STATUS",
           "KERNEL_PERSISTENT", "KERNEL_PLAIN", "library_path"]


def library_path() -> str:
    from . import build
    return build.LIB


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise NetburnError("no CUDA device: the burn runs only on the GPU")
    return torch


def _np(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def _topology(spec):
    """(kept-alive arrays, nb_topology, coeffs pointer) of a network spec."""
    arrays = dict(reac=_np(spec.reactants, np.int16), prod=_np(spec.products, np.int16),
                  coef=_np(spec.coeffs, np.float64),
                  Q=_np(getattr(spec, "Q", None), np.float64),
                  scale=_np(getattr(spec, "scale", None), np.float64),
                  ap_pg=_np(getattr(spec, "ap_pg", None), np.int8),
                  ap_coeffs=_np(getattr(spec, "ap_coeffs", None), np.float64),
                  screen=_np(getattr(spec, "screen", None), np.float64),
                  tab_of=_np(getattr(spec, "tab_of", None), np.int32),
                  tab_dens=_np(getattr(spec, "tab_dens", None), np.float64),
                  tab_t9=_np(getattr(spec, "tab_t9", None), np.float64),
                  tab_lnl=_np(getattr(spec, "tab_lnl", None), np.float64),
                  charge=_np(getattr(spec, "charge", None), np.float64))
    p = lambda a: None if a is None else a.ctypes.data
    topo = _abi.Topology(int(spec.N), int(spec.R), p(arrays["reac"]), p(arrays["prod"]),
                         p(arrays["Q"]), p(arrays["scale"]), int(bool(spec.self_heating)),
                         p(arrays["ap_pg"]), p(arrays["ap_coeffs"]), p(arrays["screen"]),
                         p(arrays["tab_of"]),
                         0 if arrays["tab_dens"] is None else arrays["tab_dens"].size,
                         0 if arrays["tab_t9"] is None else arrays["tab_t9"].size,
                         p(arrays["tab_dens"]), p(arrays["tab_t9"]), p(arrays["tab_lnl"]),
                         p(arrays["charge"]))
    return arrays, topo, p(arrays["coef"])


def specialized_source(spec, variant: int = 0) -> str:
    """CUDA source of the network-specialised burn kernel (host only)."""
    lib = _abi.load()
    arrays, topo, coef = _topology(spec)
    n = C.c_int64()
    lib.nb_specialize_source(C.byref(topo), coef, int(variant), None, 0, C.byref(n))
    buf = C.create_string_buffer(n.value + 1)
    _abi.check(lib.nb_specialize_source(C.byref(topo), coef, int(variant), buf,
                                        n.value + 1, C.byref(n)), "nb_specialize_source")
    return buf.value.decode()


def specialize_compile(spec, variant: int = 0) -> str:
    """Compile the specialised kernel for sm_103a without a GPU; returns the
    compiler log (registers, spills).  Raises NetburnError on failure."""
    lib = _abi.load()
    arrays, topo, coef = _topology(spec)
    log = C.create_string_buffer(1 << 16)
    rc = lib.nb_specialize_compile(C.byref(topo), coef, int(variant), log, len(log))
    if rc != _abi.NB_OK:
        raise NetburnError("nb_specialize_compile: " + log.value.decode(errors="replace"))
    return log.value.decode(errors="replace")


class Network:
    """A compiled network on the current CUDA device.

    ``spec`` has attributes N, R, reactants [R,3], products [R,3] (int,
    -1 padded), coeffs [R,7], Q [R] or None, scale [R] or None and
    self_heating."""

    def __init__(self, spec):
        _torch()
        lib = _abi.load()
        self.N = int(spec.N)
        self.R = int(spec.R)
        self.self_heating = bool(spec.self_heating)
        self._arrays, topo, coef = _topology(spec)
        self.has_energy = getattr(spec, "Q", None) is not None
        h = C.c_void_p()
        _abi.check(lib.nb_net_load(C.byref(topo), coef, C.byref(h)), "nb_net_load")
        self._h = h
        self.n = self.N + (1 if self.self_heating else 0)

    @property
    def handle(self):
        if self._h is None:
            raise NetburnError("network was freed")
        return self._h

    def info(self) -> dict:
        lib = _abi.load()
        out = _abi.NetInfo()
        _abi.check(lib.nb_net_get_info(self.handle, C.byref(out)), "nb_net_get_info")
        return {name: getattr(out, name) for name, _ in out._fields_
                if name != "reserved"}

    def specialize(self, variant: int = 0) -> str:
        """Build the network-specialised kernel now (nb_net_specialize);
        returns the compiler log."""
        log = C.create_string_buffer(1 << 16)
        rc = _abi.load().nb_net_specialize(self.handle, int(variant), log, len(log))
        if rc != _abi.NB_OK:
            raise NetburnError("nb_net_specialize: " + log.value.decode(errors="replace"))
        return log.value.decode(errors="replace")

    def close(self):
        if getattr(self, "_h", None) is not None:
            _abi.load().nb_net_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BurnResult(NamedTuple):
    Y: "object"
    T9: "object"
    E: "object"
    counters: "object"
    status: "object"


def _options(kernel, threads_per_block, blocks_per_sm, blob_in_shared,
             max_attempts, ws_in_shared=-1, time_budget_s=0.0, schedule=None,
             specialize=0, warps_per_zone=0):
    o = _abi.Options()
    _abi.load().nb_default_options(C.byref(o))
    if isinstance(kernel, str):
        kernel = {"auto": _abi.KERNEL_AUTO, "persistent": KERNEL_PERSISTENT,
                  "plain": KERNEL_PLAIN, "coop": KERNEL_COOP}[kernel]
    o.kernel = int(kernel)
    o.threads_per_block = int(threads_per_block)
    o.blocks_per_sm = int(blocks_per_sm)
    o.blob_in_shared = int(blob_in_shared)
    o.max_attempts = int(max_attempts)
    o.ws_in_shared = int(ws_in_shared)
    o.time_budget_s = float(time_budget_s)
    if schedule is not None:
        o.schedule = {"fifo": 0, "longest_first": 1}.get(schedule, schedule)
    o.specialize = {"auto": 0, "generic": -1, None: 0}.get(specialize, specialize)
    o.warps_per_zone = int(warps_per_zone)
    return o


def _dev(t, torch, name, shape=None):
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise NetburnError(f"{name} must be a CUDA float64 tensor")
    if not t.is_contiguous():
        raise NetburnError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise NetburnError(f"{name} has shape {tuple(t.shape)}, expected {shape}")
    return t


def burn(net: Network, Y0, T9, rho, t_end: float, rtol: float, atol: float,
         ln_mult=None, *, kernel="persistent", tape: "Optional[Tape]" = None,
         threads_per_block=0, blocks_per_sm=0, blob_in_shared=-1,
         ws_in_shared=-1, max_attempts=500000, time_budget_s=0.0, schedule=None,
         specialize=0, zeta=None, warps_per_zone=0, stream=None,
         out: Optional[BurnResult] = None):
    """Burn Z zones on the GPU.  Y0 [Z,N], T9 [Z], rho [Z] CUDA float64;
    t_end a number, or a CUDA float64 tensor [Z] of per-zone end times;
    ln_mult None, [R] or [Z,R].  specialize: 0/"auto" the kernel generated
    for the network when it qualifies, -1/"generic" the generic kernel, 1..3
    a specialised storage variant.  zeta: None or a CUDA float64 tensor [Z]
    of per-zone plasma parameters (weak screening of a screened network).
    warps_per_zone (kernel "coop"): 1, or 2 or 4 warps of one block per
    zone.  Returns BurnResult of CUDA tensors."""
    torch = _torch()
    Z = int(Y0.shape[0]) if Y0.dim() == 2 else 0
    _dev(Y0, torch, "Y0", (Z, net.N))
    _dev(T9, torch, "T9", (Z,))
    _dev(rho, torch, "rho", (Z,))
    per_zone = 0
    if ln_mult is not None:
        _dev(ln_mult, torch, "ln_mult")
        if ln_mult.dim() == 2:
            per_zone = 1
            if tuple(ln_mult.shape) != (Z, net.R):
                raise NetburnError("ln_mult must be [R] or [Z, R]")
        elif tuple(ln_mult.shape) != (net.R,):
            raise NetburnError("ln_mult must be [R] or [Z, R]")
    dev = Y0.device
    if out is None:
        out = BurnResult(torch.empty((Z, net.N), dtype=torch.float64, device=dev),
                         torch.empty((Z,), dtype=torch.float64, device=dev),
                         torch.empty((Z,), dtype=torch.float64, device=dev),
                         torch.empty((Z, NCOUNT), dtype=torch.int32, device=dev),
                         torch.empty((Z,), dtype=torch.int32, device=dev))
    o = _options(kernel, threads_per_block, blocks_per_sm, blob_in_shared,
                 max_attempts, ws_in_shared, time_budget_s, schedule, specialize,
                 warps_per_zone)
    if isinstance(t_end, torch.Tensor):
        # operator split: every zone burns for its own step
        _dev(t_end, torch, "t_end", (Z,))
        o.t_end_zone = t_end.data_ptr()
        t_end = 0.0
    if zeta is not None:
        _dev(zeta, torch, "zeta", (Z,))
        o.zeta_zone = zeta.data_ptr()
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    lib = _abi.load()
    ptr = lambda t: None if t is None else t.data_ptr()
    rc = lib.nb_burn_batch(net.handle, Z, ptr(Y0), ptr(T9), ptr(rho),
                           float(t_end), float(rtol), float(atol), ptr(ln_mult),
                           per_zone, ptr(out.Y), ptr(out.T9), ptr(out.E),
                           ptr(out.counters), ptr(out.status), C.byref(o),
                           None if tape is None else tape.handle,
                           C.c_void_p(st.cuda_stream))
    _abi.check(rc, "nb_burn_batch")
    if tape is not None:
        tape._recorded(Z, ln_mult, float(t_end), float(rtol), float(atol))
    return out


def zone_costs(net: Network, Y0, T9, rho, t_end, rtol, atol, *, zeta=None, stream=None):
    """Predicted cost of burning each zone (``nb_zone_costs``), a CUDA
    float64 tensor [Z]: the weights ``parallel.shard`` balances."""
    torch = _torch()
    Z = int(Y0.shape[0])
    _dev(Y0, torch, "Y0", (Z, net.N))
    _dev(T9, torch, "T9", (Z,))
    _dev(rho, torch, "rho", (Z,))
    cost = torch.empty(Z, dtype=torch.float64, device=Y0.device)
    o = _options("persistent", 0, 0, -1, 500000)
    if isinstance(t_end, torch.Tensor):
        _dev(t_end, torch, "t_end", (Z,))
        o.t_end_zone = t_end.data_ptr()
        t_end = 0.0
    if zeta is not None:
        _dev(zeta, torch, "zeta", (Z,))
        o.zeta_zone = zeta.data_ptr()
    st = stream if stream is not None else torch.cuda.current_stream(Y0.device)
    _abi.check(_abi.load().nb_zone_costs(net.handle, Z, Y0.data_ptr(), T9.data_ptr(),
                                         rho.data_ptr(), float(t_end), float(rtol), float(atol),
                                         C.byref(o), cost.data_ptr(), C.c_void_p(st.cuda_stream)),
               "nb_zone_costs")
    return cost


def burn_multi(sets, t_end: float, rtol: float, atol: float, *, threads_per_block=0,
               blocks_per_sm=0, max_attempts=500000, time_budget_s=0.0, stream=None):
    """Burn several networks' zones in one launch (``nb_burn_multi``).

    ``sets``: a list of dicts with keys net, Y0, T9, rho and optionally
    ln_mult ([R] or [Z, R]), t_end (a CUDA float64 tensor [Z] of per-zone
    end times) and zeta ([Z] plasma parameters); tensors as for ``burn``.  Returns one BurnResult per set."""
    torch = _torch()
    if not 1 <= len(sets) <= _abi.MULTI_MAX_SETS:
        raise NetburnError(f"1..{_abi.MULTI_MAX_SETS} sets")
    arr = (_abi.BurnSet * len(sets))()
    outs = []
    ptr = lambda t: None if t is None else t.data_ptr()
    for b, d in zip(arr, sets):
        net = d["net"]
        Y0, T9, rho = d["Y0"], d["T9"], d["rho"]
        Z = int(Y0.shape[0])
        _dev(Y0, torch, "Y0", (Z, net.N))
        _dev(T9, torch, "T9", (Z,))
        _dev(rho, torch, "rho", (Z,))
        lm = d.get("ln_mult")
        per_zone = 0
        if lm is not None:
            _dev(lm, torch, "ln_mult")
            per_zone = 1 if lm.dim() == 2 else 0
            if tuple(lm.shape) not in ((net.R,), (Z, net.R)):
                raise NetburnError("ln_mult must be [R] or [Z, R]")
        tz = d.get("t_end")
        if tz is not None:
            _dev(tz, torch, "t_end", (Z,))
        zt = d.get("zeta")
        if zt is not None:
            _dev(zt, torch, "zeta", (Z,))
        dev = Y0.device
        out = BurnResult(torch.empty((Z, net.N), dtype=torch.float64, device=dev),
                         torch.empty((Z,), dtype=torch.float64, device=dev),
                         torch.empty((Z,), dtype=torch.float64, device=dev),
                         torch.empty((Z, NCOUNT), dtype=torch.int32, device=dev),
                         torch.empty((Z,), dtype=torch.int32, device=dev))
        outs.append(out)
        b.net = net.handle.value
        b.Z = Z
        b.Y0, b.T9_0, b.rho = ptr(Y0), ptr(T9), ptr(rho)
        b.ln_mult, b.ln_mult_per_zone, b.t_end_zone = ptr(lm), per_zone, ptr(tz)
        b.zeta_zone = ptr(zt)
        b.Y, b.T9, b.E = ptr(out.Y), ptr(out.T9), ptr(out.E)
        b.counters, b.status = ptr(out.counters), ptr(out.status)
    o = _options("persistent", threads_per_block, blocks_per_sm, -1, max_attempts,
                 time_budget_s=time_budget_s)
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = _abi.load().nb_burn_multi(len(sets), arr, float(t_end), float(rtol), float(atol),
                                   C.byref(o), C.c_void_p(st.cuda_stream))
    _abi.check(rc, "nb_burn_multi")
    return outs


class BurnGraph:
    """A burn captured once in a CUDA graph and replayed.

    The tensors passed here are the graph's inputs: write new zone data into
    them in place (same shapes) and call ``replay()``; ``out`` holds the
    results.  Capture happens after one ordinary burn with the same launch
    options, so the device workspace is already allocated and the captured
    work is one counter reset and one kernel launch."""

    def __init__(self, net: "Network", Y0, T9, rho, t_end, rtol, atol,
                 ln_mult=None, **launch):
        torch = _torch()
        self.args = (net, Y0, T9, rho, t_end, rtol, atol, ln_mult)
        self.launch = launch
        self.out = burn(*self.args, **launch)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            burn(*self.args, out=self.out, **launch)
        torch.cuda.synchronize()

    def replay(self) -> "BurnResult":
        self.graph.replay()
        return self.out


def burn_host(net: Network, Y0, T9, rho, t_end, rtol, atol, ln_mult=None, *,
              kernel="persistent", threads_per_block=0, blocks_per_sm=0,
              blob_in_shared=-1, ws_in_shared=-1, max_attempts=500000,
              specialize=0, zeta=None, stream=None, out=None):
    """Burn from host (numpy) arrays through ``nb_burn_batch_host``: the
    library copies the inputs in, burns and copies the outputs back.
    Returns a dict of numpy arrays; ``out`` may supply preallocated (e.g.
    pinned) output arrays."""
    torch = _torch()
    Y0 = _np(Y0, np.float64)
    Z = Y0.shape[0]
    T9 = _np(T9, np.float64)
    rho = _np(rho, np.float64)
    lm = _np(ln_mult, np.float64)
    per_zone = 1 if (lm is not None and lm.ndim == 2) else 0
    if out is None:
        out = dict(Y=np.empty((Z, net.N)), T9=np.empty(Z), E=np.empty(Z),
                   counters=np.empty((Z, NCOUNT), np.int32),
                   status=np.empty(Z, np.int32))
    o = _options(kernel, threads_per_block, blocks_per_sm, blob_in_shared,
                 max_attempts, ws_in_shared, specialize=specialize)
    if zeta is not None:
        # per-zone plasma parameters: a device array, as for nb_burn_batch
        _dev(zeta, torch, "zeta", (Z,))
        o.zeta_zone = zeta.data_ptr()
    st = stream if stream is not None else torch.cuda.current_stream()
    p = lambda a: None if a is None else a.ctypes.data
    rc = _abi.load().nb_burn_batch_host(
        net.handle, Z, p(Y0), p(T9), p(rho), float(t_end), float(rtol),
        float(atol), p(lm), per_zone, p(out["Y"]), p(out["T9"]), p(out["E"]),
        p(out["counters"]), p(out["status"]), C.byref(o),
        C.c_void_p(st.cuda_stream))
    _abi.check(rc, "nb_burn_batch_host")
    return out


class Tape:
    """Device record of a burn's accepted steps, for ``adjoint``: the schedule
    of every step and the states at checkpoints every ``ckpt_stride`` steps
    (0: the library default; 1: every state)."""

    def __init__(self, net: Network, Z: int, max_steps: int, ckpt_stride: int = 0):
        _torch()
        self.net = net
        self.Z = int(Z)
        self.max_steps = int(max_steps)
        self.ckpt_stride = int(ckpt_stride)
        h = C.c_void_p()
        _abi.check(_abi.load().nb_tape_alloc(net.handle, self.Z, self.max_steps,
                                             self.ckpt_stride, C.byref(h)), "nb_tape_alloc")
        self._h = h
        self.recorded = None

    @property
    def handle(self):
        if self._h is None:
            raise NetburnError("tape was freed")
        return self._h

    def read(self, z: int) -> dict:
        """Zone z's record (``nb_tape_read``): numpy arrays t, h, k (order)
        and x [S+1, n], E [S+1] (NaN where the tape keeps no state), record 0
        the initial point."""
        cap = self.max_steps + 1
        n = self.net.n
        t = np.empty(cap)
        h = np.empty(cap)
        k = np.empty(cap, np.int32)
        x = np.empty((cap, n))
        E = np.empty(cap)
        cnt = C.c_int32(0)
        _abi.check(_abi.load().nb_tape_read(self.handle, int(z), cap, t.ctypes.data,
                                            h.ctypes.data, k.ctypes.data, x.ctypes.data,
                                            E.ctypes.data, C.byref(cnt)), "nb_tape_read")
        c = cnt.value
        return dict(t=t[:c].copy(), h=h[:c].copy(), k=k[:c].copy(), x=x[:c].copy(),
                    E=E[:c].copy())

    def _recorded(self, Z, ln_mult, t_end, rtol, atol):
        self.recorded = dict(Z=Z, per_zone=(ln_mult is not None and ln_mult.dim() == 2),
                             t_end=t_end, rtol=rtol, atol=atol)

    def close(self):
        if getattr(self, "_h", None) is not None:
            _abi.load().nb_tape_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def adjoint(net: Network, tape: Tape, gY, gE=None, gT9=None, *, stream=None,
            want_initial=True, kernel="auto", threads_per_block=0, blocks_per_sm=0,
            ws_in_shared=-1, blob_in_shared=-1):
    """Discrete adjoint of the burn recorded on ``tape``.  gY [K,Z,N], gE and
    gT9 [K,Z] (or None).  kernel: "auto" (on a checkpointed tape the
    arithmetic of the burn that recorded it; at stride 1 one warp per zone
    for networks of 24 or more state entries), "persistent" (one lane per
    zone) or "coop" (one warp per zone); on a checkpointed tape an explicit
    kernel must match the recording burn's.  Returns (d_ln_mult [K,Z,R],
    dY0 [K,Z,N], dT0 [K,Z])."""
    torch = _torch()
    if tape.recorded is None:
        raise NetburnError("tape holds no burn")
    Z = tape.recorded["Z"]
    if gY.dim() == 2:
        gY = gY.unsqueeze(0)
    K = int(gY.shape[0])
    _dev(gY, torch, "gY", (K, Z, net.N))
    if gE is not None:
        gE = gE.reshape(K, Z).contiguous()
        _dev(gE, torch, "gE", (K, Z))
    if gT9 is not None:
        gT9 = gT9.reshape(K, Z).contiguous()
        _dev(gT9, torch, "gT9", (K, Z))
    dev = gY.device
    dl = torch.empty((K, Z, net.R), dtype=torch.float64, device=dev)
    dY0 = torch.empty((K, Z, net.N), dtype=torch.float64, device=dev) if want_initial else None
    dT0 = torch.empty((K, Z), dtype=torch.float64, device=dev) if want_initial else None
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    ptr = lambda t: None if t is None else t.data_ptr()
    o = None
    if (kernel, threads_per_block, blocks_per_sm, ws_in_shared, blob_in_shared) != \
            ("auto", 0, 0, -1, -1):
        o = _options(kernel, threads_per_block, blocks_per_sm, blob_in_shared, 500000,
                     ws_in_shared)
    rc = _abi.load().nb_burn_adjoint_ex(net.handle, tape.handle, K, ptr(gY), ptr(gE),
                                        ptr(gT9), ptr(dl), ptr(dY0), ptr(dT0),
                                        None if o is None else C.byref(o),
                                        C.c_void_p(st.cuda_stream))
    _abi.check(rc, "nb_burn_adjoint_ex")
    return dl, dY0, dT0


def _autograd():
    import torch

    class Burn(torch.autograd.Function):
        """(Y0, T9, rho, ln_mult) -> (Y, T9, E, counters, status) with a
        discrete-adjoint backward (counters and status are not
        differentiable).  ln_mult may be [R] (shared) or [Z, R]; its gradient is
        d/d ln(rate multiplier) of every reaction."""

        @staticmethod
        def forward(ctx, Y0, T9, rho, ln_mult, net, t_end, rtol, atol,
                    max_steps=20000):
            Z = Y0.shape[0]
            lm = None
            if ln_mult is not None:
                lm = ln_mult.detach().contiguous()
            tape = Tape(net, Z, max_steps)
            out = burn(net, Y0.detach().contiguous(), T9.detach().contiguous(),
                       rho.detach().contiguous(), t_end, rtol, atol, lm, tape=tape)
            ctx.tape = tape
            ctx.net = net
            ctx.shared = ln_mult is not None and ln_mult.dim() == 1
            ctx.has_mult = ln_mult is not None
            ctx.mark_non_differentiable(out.counters, out.status)
            return out.Y, out.T9, out.E, out.counters, out.status

        @staticmethod
        def backward(ctx, gY, gT9, gE, _gc, _gs):
            net = ctx.net
            torch_ = torch
            Z = gY.shape[0] if gY is not None else ctx.tape.recorded["Z"]
            dev = gY.device if gY is not None else gT9.device
            if gY is None:
                gY = torch_.zeros((Z, net.N), dtype=torch_.float64, device=dev)
            dl, dY0, dT0 = adjoint(net, ctx.tape, gY.contiguous().unsqueeze(0),
                                   None if gE is None else gE.contiguous().unsqueeze(0),
                                   None if gT9 is None else gT9.contiguous().unsqueeze(0))
            dl, dY0, dT0 = dl[0], dY0[0], dT0[0]
            g_lm = None
            if ctx.has_mult:
                g_lm = dl.sum(0) if ctx.shared else dl
            return dY0, dT0, None, g_lm, None, None, None, None, None

    return Burn


class _LazyBurn:
    _cls = None

    def __getattr__(self, name):
        if _LazyBurn._cls is None:
            _LazyBurn._cls = _autograd()
        return getattr(_LazyBurn._cls, name)


Burn = _LazyBurn()
