#!/usr/bin/env python
"""Zone-burns per second of the batched stiff reaction-network burn on GB300.

One step = one burn of the whole workload: every zone of the self-heating
13-species alpha chain (65,536 zones, T9 log-uniform [0.5, 5], rho
log-uniform [1e5, 1e8], t_end 1e-3 s, rtol 1e-8, atol 1e-12) integrated by
the persistent lane-per-zone kernel, inputs already in HBM.  Prints one JSON
line (rank 0).  ``--impl reference`` times the CPU oracle instead.

Multi-GPU: one process per GPU (torchrun); every rank burns its own zones
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = ("zone-burns/sec (FP64, rtol=1e-8) and adjoint gradients/sec vs plain "
          "GPU launch & CPU oracle")
WORKLOAD = "chain13_heat"
WORKLOAD_DESC = ("13-species alpha chain with self-heating (12 rates, Q~U[1,10]), "
                 "65536 zones, T9 log-U[0.5,5], rho log-U[1e5,1e8], Y0=1/4, "
                 "t_end 1e-3 s, rtol 1e-8, atol 1e-12")


# The other workloads of the configuration table, each a sub-entry of the
# line (name, zones, options of config_entry): the fixed-temperature chain,
# the 48-species network at its full 262,144 zones, and the 128-species
# self-heating network on a seeded 1,024-zone prefix of its zones, with a
# watchdog (by default), or at its full 131,072 zones ("cfg4_full", about
# eight minutes).  The 128-species network runs two warps per zone: on the
# prefix one warp gave 170 zone-burns/s, two 275, four 86.  The sensitivity
# workload is the "adjoint" entry.
CFG4_LAUNCH = dict(kernel="coop", warps_per_zone=2)
CONFIG_TABLE = {
    "cfg0": ("chain13", None, dict(cpu_zones=4096)),
    "cfg2": ("net48", None, dict(cpu_zones=256)),
    "cfg4": ("net128_heat", 1024, dict(cpu_zones=16, plain_zones=0, steps=1, warmup=0,
                                       budget_s=60.0, launch=CFG4_LAUNCH,
                                       full_zones=131072)),
    "cfg4_full": ("net128_heat", 131072, dict(cpu_zones=0, plain_zones=0, steps=1, warmup=0,
                                              launch=CFG4_LAUNCH)),
}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# the sources that determine the timed kernel's code: the integrator, the
# exp, the compiled-network layout, the generic network walk and the code
# generator of the specialised kernel, and the launch code
KERNEL_SOURCES = ("integrator.cuh", "expf64.cuh", "blob.h", "device.cuh", "netload.cpp",
                  "codegen.cpp", "burn.cu", "coop.cuh", "adjoint.cuh", "adjoint.cu")


def _code_only(text: str) -> str:
    """C++ source without its comments and blank lines (what a comment edit
    leaves unchanged).  Text after a // inside a string literal goes too; in
    these sources that is only the text of generated comments."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*", "", line).rstrip() for line in text.splitlines())
    return "\n".join(line for line in lines if line)


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2312_02836_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(d, f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def launch_shape(launch, variant):
    """lanes per SM and specialised variant of a persistent launch (what sets
    the lanes in flight and the code of the kernel); None with shared-memory
    work arrays, which the profile does not cover."""
    if launch.get("ws_in_shared", -1) > 0:
        return None
    return "%d,%d" % ((launch.get("threads_per_block", 0) or 128) *
                      (launch.get("blocks_per_sm", 0) or 1), variant)


def coop_shape(launch):
    """threads per block, blocks per SM and warps per zone of a warp-kernel
    launch (which instance runs and how many share an SM); None for the other
    kernels, whose entries do not check the shape."""
    if launch.get("kernel") != "coop":
        return None
    return "coop,%d,%d,%d" % (launch.get("threads_per_block", 0) or 0,
                              launch.get("blocks_per_sm", 0) or 0,
                              launch.get("warps_per_zone", 0) or 0)


def profiled_traffic(kernel, Z, shape, workload="chain13_heat"):
    """DRAM bytes per launch from the committed ncu summary of this kernel on
    this workload, or None when the kernel sources, the zone count or the
    launch shape (None: not checked) differ from the profiled ones."""
    path = os.path.join(ROOT, "profiles", kernel + "_" + workload + ".md")
    if not os.path.exists(path):
        return None
    # one block of "key: value" lines per profiled launch shape, each opened
    # by a line that starts with "machine-readable"
    blocks, kv = [], None
    for line in open(path):
        if line.startswith("machine-readable"):
            kv = {}
            blocks.append(kv)
        elif kv is not None and ":" in line and not line.startswith(("|", "#", " ")):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    for kv in blocks:
        if (kv.get("source_hash") == kernel_source_hash() and kv.get("zones") == str(Z)
                and (shape is None or kv.get("launch") == shape)
                and "dram_bytes_per_launch" in kv):
            return int(kv["dram_bytes_per_launch"])
    return None


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names[1:], parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def zone_bytes(N: int) -> int:
    """Algorithmic HBM bytes per zone-burn: Y0, T9, rho in; Y, T9, E, nine
    int32 counters and the status out."""
    return 16 * N + 8 * 4 + 9 * 4 + 4


def workload_desc(name: str, Z: int) -> str:
    c = gen.CONFIGS[name]
    net = gen.network(name)
    return (f"{name}: {net.N} species / {net.R} rates, {'self-heating' if c['heat'] else 'fixed T'}, "
            f"{Z} zones, T9 log-U{list(c['T9'])}, rho log-U{list(c['rho'])}, t_end {c['t_end']}, "
            f"rtol {c['rtol']}, atol {c['atol']}")


def sampled_parity(name, net, z, s, out, n) -> dict:
    """The GPU result of this very launch against the oracle on a seeded
    sample of its zones (tests/parity.py bar, its measured part from the
    oracle's rounding variants on the same sample)."""
    import oracle
    from tests.parity import compare, oracle_spread, to_numpy
    Z = z["T9"].shape[0]
    sel = np.unique(np.random.default_rng(12345).choice(Z, min(n, Z), replace=False))
    run = lambda v: oracle.burn(net, z["Y"][sel], z["T9"][sel], z["rho"][sel], s["t_end"],
                                s["rtol"], s["atol"],
                                zeta=z["zeta"][sel] if "zeta" in z else None, variant=v)
    o = run(0)
    spread = oracle_spread(o, [run(v) for v in oracle.VARIANTS], s["atol"], s["rtol"])
    g = {k: v[sel] for k, v in to_numpy(out).items()}
    fin = g["status"] != 6          # zones the watchdog stopped are not compared
    if not fin.all():
        g = {k: v[fin] for k, v in g.items()}
        o = {k: (v[fin] if isinstance(v, np.ndarray) else v) for k, v in o.items()}
        spread = dict(spread, status_sensitive=spread["status_sensitive"][fin])
    try:
        rep = compare(g, o, s["atol"], rtol=s["rtol"], spread=spread)
        rep["passed"] = True
    except AssertionError as e:
        rep = {"passed": False, "error": str(e)[:300]}
    rep["sample"] = int(sel.size)
    rep["compared_finished"] = int(fin.sum())
    return rep


def cpu_baseline(name: str, Z_sample: int, zone_offset: int = 0, threads: int = 0) -> dict:
    """The oracle, as it stands, on a bounded sample of the workload (all host
    cores, or `threads` of them)."""
    import oracle
    net, z, s = gen.problem(name, zone_offset + Z_sample)
    z = {k: v[zone_offset:] for k, v in z.items()}
    t0 = time.perf_counter()
    out = oracle.burn(net, z["Y"], z["T9"], z["rho"], s["t_end"], s["rtol"], s["atol"],
                      zeta=z.get("zeta"), threads=threads)
    dt = time.perf_counter() - t0
    return {"value": Z_sample / dt, "unit": "zone-burns/s", "cores": int(out["threads"]),
            "kind": "oracle", "seconds": dt,
            "sample": f"first {Z_sample} zones of {name} (i.i.d. seeded zones), "
                      + ("all host cores" if not threads else f"{threads} host core(s)")}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    Zs = args.ref_zones
    for _ in range(args.warmup):
        cpu_baseline(WORKLOAD, max(64, Zs // 16))
    times = []
    cores = 0
    for k in range(args.steps):
        r = cpu_baseline(WORKLOAD, Zs, zone_offset=k * Zs)
        times.append(r["seconds"])
        cores = r["cores"]
    per = statistics.mean(times)
    value = Zs / per
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "zone-burns/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "zones_per_step": Zs},
            "cpu_baseline": {"value": value, "unit": "zone-burns/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{Zs} zones of the workload per step"},
            "e2e": {"value": value, "unit": "zone-burns/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_native(args):
    import torch
    import paper_2312_02836_gb300 as nb
    from paper_2312_02836_gb300 import metrics

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    workload = args.workload
    Z = args.zones or gen.CONFIGS[workload]["Z"]
    Z_job = Z * ws
    net_spec, zall, s = gen.problem(workload, Z_job)
    if args.t_end is not None:
        s["t_end"] = args.t_end
    from paper_2312_02836_gb300.parallel import max_over_ranks, shard
    netc = nb.Network(net_spec)
    # weak scaling: Z zones per rank on average, the ranges balanced by each
    # zone's predicted cost (every rank predicts all zones, the same numbers)
    cost = None
    if ws > 1:
        ca = {k: torch.from_numpy(v).to(dev) for k, v in zall.items()}
        cost = nb.zone_costs(netc, ca["Y"], ca["T9"], ca["rho"], s["t_end"], s["rtol"],
                             s["atol"], zeta=ca.get("zeta")).cpu().numpy()
        del ca
    lo, hi = shard(Z_job, ws, rank, cost)
    z = {k: np.ascontiguousarray(v[lo:hi]) for k, v in zall.items()}
    Z = hi - lo
    info = netc.info()
    Y0 = torch.from_numpy(z["Y"]).to(dev)
    T9 = torch.from_numpy(z["T9"]).to(dev)
    rho = torch.from_numpy(z["rho"]).to(dev)
    # a screened workload's per-zone plasma parameter, given to every burn
    zk = dict(zeta=torch.from_numpy(z["zeta"]).to(dev)) if "zeta" in z else {}
    out = None
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()

    if (args.blocks_per_sm or args.threads_per_block or args.ws_in_shared >= 0 or args.no_autotune
            or args.specialize is not None or args.kernel != "persistent"):
        launch = dict(blocks_per_sm=args.blocks_per_sm,
                      threads_per_block=args.threads_per_block,
                      ws_in_shared=args.ws_in_shared,
                      specialize=0 if args.specialize is None else args.specialize)
        if args.kernel != "persistent":
            launch["kernel"] = args.kernel
            if args.warps_per_zone:
                launch["warps_per_zone"] = args.warps_per_zone
        tune_ms = None
    else:
        from paper_2312_02836_gb300.autotune import autotune
        launch = autotune(netc, Y0, T9, rho, s["t_end"], s["rtol"], s["atol"], extra=zk)
        tune_ms = launch.pop("_timings_ms")

    def step(kernel=None):
        nonlocal out
        opts = dict(launch) if kernel is None else dict(kernel=kernel)
        out = nb.burn(netc, Y0, T9, rho, s["t_end"], s["rtol"], s["atol"], out=out,
                      **opts, **zk)

    for _ in range(args.warmup):
        step()
    barrier()
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush.fill_(float(k))                 # L2 flush, outside the timed events
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    barrier()
    clk = clocks.stop() if clocks else None
    ms = [a.elapsed_time(b) for a, b in ev]
    local_ms = statistics.mean(ms)          # this rank's launch (its roofline)
    mean_ms = max_over_ranks(local_ms, dev)
    variant = netc.info()["last_specialized"]
    kname = ("k_burn_coop" if launch.get("kernel") == "coop" else
             "nb_spec_burn" if variant else "k_burn_persistent")
    counters = out.counters.cpu().numpy()
    status = out.status.cpu().numpy()
    ops = metrics.burn_ops(info, counters, net_spec.self_heating)
    value = Z_job / (mean_ms * 1e-3)

    # ---- end to end through the host-pointer C entry point (pinned buffers),
    # every rank its own zones, the slowest rank's time
    N = net_spec.N
    hY0 = torch.from_numpy(z["Y"]).pin_memory().numpy()
    hT9 = torch.from_numpy(z["T9"]).pin_memory().numpy()
    hrho = torch.from_numpy(z["rho"]).pin_memory().numpy()
    hout = dict(Y=torch.empty((Z, N), dtype=torch.float64).pin_memory().numpy(),
                T9=torch.empty(Z, dtype=torch.float64).pin_memory().numpy(),
                E=torch.empty(Z, dtype=torch.float64).pin_memory().numpy(),
                counters=torch.empty((Z, nb.NCOUNT), dtype=torch.int32).pin_memory().numpy(),
                status=torch.empty(Z, dtype=torch.int32).pin_memory().numpy())
    if not args.no_e2e:
        nb.burn_host(netc, hY0, hT9, hrho, s["t_end"], s["rtol"], s["atol"], out=hout,
                     **launch, **zk)
    e2e_t = []
    for _ in range(0 if args.no_e2e else max(2, min(args.steps, 5))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nb.burn_host(netc, hY0, hT9, hrho, s["t_end"], s["rtol"], s["atol"], out=hout,
                     **launch, **zk)
        e2e_t.append(time.perf_counter() - t0)
    if e2e_t:
        assert np.array_equal(hout["Y"], out.Y.cpu().numpy())
        e2e_s = max_over_ranks(statistics.mean(e2e_t), dev)
    h2d = hY0.nbytes + hT9.nbytes + hrho.nbytes
    d2h = sum(a.nbytes for a in hout.values())
    if rank != 0:
        return

    # ---- plain one-thread-per-zone launch, same inputs and tolerances
    plain_ms = []
    for k in range(0 if args.no_plain else 2):
        flush.fill_(2.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step("plain")
        b.record(stream)
        torch.cuda.synchronize()
        plain_ms.append(a.elapsed_time(b))
    plain_equal = bool(np.array_equal(out.Y.cpu().numpy(), hout["Y"])) if plain_ms and e2e_t else None

    # ---- roofline of the burn kernel (one launch per step)
    achieved = ops["flops"] / (local_ms * 1e-3) / 1e12
    peak = metrics.FP64_PEAK_TFLOPS
    traffic = profiled_traffic(kname, Z, launch_shape(launch, variant))
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": kname,
                "timed": ("CUDA events around each step: the burn kernel, 99.9 % of the "
                          "step's device time, plus the longest-first pre-pass and sort"),
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2070 MHz",
                "flops_per_launch": ops["flops"],
                "special_functions_per_launch": ops["special"],
                "algorithmic_bytes_per_launch": int(Z * zone_bytes(net_spec.N))}

    base = None
    if not args.no_cpu_baseline:
        base = cpu_baseline(workload, args.cpu_zones)
        base.pop("seconds", None)
        # and on one core, on a smaller sample of the same zones
        one = cpu_baseline(workload, max(64, args.cpu_zones // 16), threads=1)
        one.pop("seconds", None)
        base["one_core"] = one
    parity = None
    if args.sample_parity:
        parity = sampled_parity(workload, net_spec, z, s, out, args.sample_parity)

    adj = None
    if args.adjoint:
        adj = adjoint_bench(nb, torch, dev, flush, metrics)
    adj_cfg = {}
    if args.cfg4_adjoint:
        # the 128-species network's adjoint over all 600 multipliers on an
        # 8192-zone subset: every state on the tape (stride 1), so the
        # forward may run two warps per zone; zones past 4000 steps (the
        # runaways) end TAPE_FULL and get no gradient
        adj_cfg["cfg4"] = adjoint_bench(nb, torch, dev, flush, metrics, repeats=1,
                                        name="net128_heat", Z=8192, max_steps=4000, stride=1,
                                        launch=CFG4_LAUNCH, full_tape=False)
    multi = multi_bench(nb, torch, dev, flush) if args.multi else None
    configs = {}
    for cname in [c for c in args.configs.split(",") if c]:
        name, Zc, kw = CONFIG_TABLE[cname]
        sp = args.sample_parity
        configs[cname] = config_entry(nb, torch, dev, flush, metrics, name, Zc,
                                      sample_parity=sp, **kw)

    line = {"metric": METRIC, "value": value, "unit": "zone-burns/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC if workload == WORKLOAD else
                       workload_desc(workload, Z_job // ws), "zones_per_gpu": Z_job // ws,
                       "l2": "256 MiB buffer written between timed steps (L2 flush)",
                       "kernel": ("persistent warp-per-zone, device work queue, arrays in "
                                  "shared memory" if launch.get("kernel") == "coop" else
                                  "persistent lane-per-zone, device work queue, "
                                  + ("code generated for the network (storage variant %d)" % variant
                                     if variant else "generic network walk")),
                       "launch": launch,
                       "autotune_ms": None if tune_ms is None else
                       [[c, round(m, 2)] for c, m in tune_ms]},
            "roofline": roofline, "cpu_baseline": base,
            "e2e": None if not e2e_t else {"value": Z_job / e2e_s, "unit": "zone-burns/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "path": "nb_burn_batch_host (pinned host buffers, copies inside)"},
            # per step: the burn kernel, plus the longest-first pre-pass
            # (k_burn_estimate) whenever there is more than one zone; the
            # CUB sort kernels between them are library code
            "gpu_launches": args.steps * (2 if Z > 1 else 1),
            "clocks": clk,
            "plain_launch": None if not plain_ms else {
                "value": Z / (statistics.mean(plain_ms) * 1e-3),
                "unit": "zone-burns/s", "ms": statistics.mean(plain_ms),
                "bitwise_equal_to_persistent": plain_equal},
            "zones_ok": int((status == 0).sum()),
            "events": ops["events"]}
    if adj is not None:
        line["adjoint"] = adj
    if adj_cfg:
        line["adjoint_configs"] = adj_cfg
    if multi is not None:
        line["multi_network"] = multi
    if parity is not None:
        line["sampled_parity"] = parity
    if configs:
        line["configs"] = configs
    print(json.dumps(line), flush=True)


def config_entry(nb, torch, dev, flush, metrics, name, Z=None, steps=3, warmup=1,
                 sample_parity=256, cpu_zones=256, tune_zones=32768, plain_zones=16384,
                 budget_s=0.0, launch=None, full_zones=None) -> dict:
    """One workload of the configuration table at its size: zone-burns/s of
    the autotuned persistent launch (autotuned on the first tune_zones zones,
    the launch shape does not depend on the zone count once lanes are
    outnumbered), the FP64 roofline of its kernel, the plain one-thread-per-
    zone launch on a prefix of plain_zones zones, the oracle on cpu_zones
    zones of the host, and the launch's sampled parity with the oracle.
    budget_s > 0: the device watchdog ends zones still burning after that
    long (the entry then counts only finished zones).  launch: a fixed
    launch instead of the autotuner's.  full_zones: the workload's full size,
    when Z is a prefix of it: the entry projects the full burn's time from
    the prefix's flops and FP64 rate."""
    from paper_2312_02836_gb300.autotune import autotune
    net, z, s = gen.problem(name, Z)
    Z = z["T9"].shape[0]
    nc = nb.Network(net)
    info = nc.info()
    d = {k: torch.from_numpy(v).to(dev) for k, v in z.items()}
    zk = dict(zeta=d["zeta"]) if "zeta" in d else {}
    if launch is None:
        Zt = min(Z, tune_zones)
        tz = {k: v[:Zt].contiguous() for k, v in d.items()}
        launch = autotune(nc, tz["Y"], tz["T9"], tz["rho"], s["t_end"], s["rtol"], s["atol"],
                          extra=dict(zeta=tz["zeta"]) if "zeta" in tz else {},
                          key=f"{name}:{Zt}")
        tune_ms = launch.pop("_timings_ms")
    else:
        launch, tune_ms = dict(launch), []
    stream = torch.cuda.current_stream(dev)
    out = None

    def step(**extra):
        nonlocal out
        out = nb.burn(nc, d["Y"], d["T9"], d["rho"], s["t_end"], s["rtol"], s["atol"],
                      out=out, time_budget_s=budget_s, **{**launch, **extra}, **zk)

    for _ in range(warmup):
        step()
    ms = []
    for k in range(steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    mean_ms = statistics.mean(ms)
    counters = out.counters.cpu().numpy()
    status = out.status.cpu().numpy()
    done = status != 6
    ops = metrics.burn_ops(info, counters[done], net.self_heating)
    achieved = ops["flops"] / (mean_ms * 1e-3) / 1e12
    kernel = launch.get("kernel", "persistent")
    kname = {"coop": "k_burn_coop"}.get(kernel, "nb_spec_burn" if nc.info()["last_specialized"]
                                        else "k_burn_persistent")
    entry = {"workload": workload_desc(name, Z), "zones": Z,
             "value": int(done.sum()) / (mean_ms * 1e-3), "unit": "zone-burns/s",
             "ms_per_step": mean_ms, "steps": steps, "launch": launch,
             "autotune_ms": [[c, round(m, 2)] for c, m in tune_ms],
             "zones_ok": int((status == 0).sum()), "zones_timed_out": int((~done).sum()),
             "roofline": {"bound": "alu", "achieved": achieved,
                          "peak": metrics.FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                          "frac": achieved / metrics.FP64_PEAK_TFLOPS,
                          "traffic": profiled_traffic(kname, Z, coop_shape(launch), workload=name),
                          "kernel": kname, "flops_per_launch": ops["flops"],
                          "algorithmic_bytes_per_launch": int(Z * zone_bytes(net.N)),
                          "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2070 MHz"},
             "events": ops["events"]}
    if budget_s > 0:
        entry["time_budget_s"] = budget_s
    if full_zones and done.any():
        per_zone = ops["flops"] / done.sum()
        entry["projected_full_size"] = {
            "zones": full_zones, "flops": per_zone * full_zones,
            "seconds_at_this_rate": per_zone * full_zones / (achieved * 1e12),
            "seconds_at_fp64_peak": per_zone * full_zones / (metrics.FP64_PEAK_TFLOPS * 1e12),
            "basis": f"mean algorithmic flops of the {int(done.sum())} finished zones of a "
                     f"{Z}-zone seeded prefix"}
    if plain_zones:
        Zp = min(Z, plain_zones)
        pz = {k: v[:Zp].contiguous() for k, v in d.items()}
        pzk = dict(zeta=pz["zeta"]) if "zeta" in pz else {}
        nb.burn(nc, pz["Y"], pz["T9"], pz["rho"], s["t_end"], s["rtol"], s["atol"],
                kernel="plain", time_budget_s=budget_s, **pzk)
        flush.fill_(5.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        po = nb.burn(nc, pz["Y"], pz["T9"], pz["rho"], s["t_end"], s["rtol"], s["atol"],
                     kernel="plain", time_budget_s=budget_s, **pzk)
        b.record(stream)
        torch.cuda.synchronize()
        pdone = int((po.status.cpu().numpy() != 6).sum())
        entry["plain_launch"] = {"value": pdone / (a.elapsed_time(b) * 1e-3),
                                 "unit": "zone-burns/s", "zones": Zp}
    if sample_parity:
        entry["sampled_parity"] = sampled_parity(name, net, z, s, out, sample_parity)
    if cpu_zones:
        base = cpu_baseline(name, cpu_zones)
        base.pop("seconds", None)
        entry["cpu_baseline"] = base
    return entry


def adjoint_bench(nb, torch, dev, flush, metrics, repeats=3, name="net48_adjoint", Z=None,
                  max_steps=4000, stride=16, launch=None, full_tape=True) -> dict:
    """Adjoint gradients/s: the sensitivity workload (by default the
    48-species one), 6 cotangents per zone (energy + the 5 largest final
    abundances), forward with tape plus reverse sweep (which recomputes the
    checkpointed blocks at stride > 1), timed `repeats` times, with the FP64
    roofline of the reverse kernel.  A zone that needs more than max_steps
    steps ends TAPE_FULL and gets no gradient (counted)."""
    net, z, s = gen.problem(name, Z)
    Z = z["T9"].shape[0]
    nc = nb.Network(net)
    info = nc.info()
    Y0 = torch.from_numpy(z["Y"]).to(dev)
    T9 = torch.from_numpy(z["T9"]).to(dev)
    rho = torch.from_numpy(z["rho"]).to(dev)
    # one warp per zone for a large network, forward and reverse (a
    # checkpointed tape is recomputed in the arithmetic that recorded it)
    fk = "coop" if info["n_state"] >= 24 else "persistent"
    kname = "k_adjoint_coop" if fk == "coop" else "k_adjoint"
    fl = dict(kernel=fk) if launch is None else dict(launch)
    tape = nb.Tape(nc, Z, max_steps, stride)
    fw = nb.burn(nc, Y0, T9, rho, s["t_end"], s["rtol"], s["atol"], tape=tape, **fl)
    torch.cuda.synchronize()
    Yf = fw.Y.cpu().numpy()
    top = gen.largest_species(Yf, 5)
    K = 6
    gY = np.zeros((K, Z, net.N))
    gE = np.zeros((K, Z))
    gE[0] = 1.0
    for q in range(5):
        gY[q + 1, np.arange(Z), top[:, q]] = 1.0
    gYd = torch.from_numpy(gY).to(dev)
    gEd = torch.from_numpy(gE).to(dev)
    nb.adjoint(nc, tape, gYd, gEd)
    torch.cuda.synchronize()
    fwd, rev = [], []
    for k in range(repeats):
        flush.fill_(3.0 + k)
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record()
        fw = nb.burn(nc, Y0, T9, rho, s["t_end"], s["rtol"], s["atol"], tape=tape, **fl)
        b.record()
        nb.adjoint(nc, tape, gYd, gEd)
        c.record()
        torch.cuda.synchronize()
        fwd.append(a.elapsed_time(b))
        rev.append(b.elapsed_time(c))
    fwd_ms, adj_ms = statistics.mean(fwd), statistics.mean(rev)
    # the same with every state on the tape (stride 1): no recomputation
    full_ms = None
    if full_tape and stride != 1:
        full = nb.Tape(nc, Z, max_steps, 1)
        nb.burn(nc, Y0, T9, rho, s["t_end"], s["rtol"], s["atol"], tape=full, **fl)
        flush.fill_(9.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        nb.adjoint(nc, full, gYd, gEd)
        b.record()
        torch.cuda.synchronize()
        full_ms = a.elapsed_time(b)
        del full
    st = fw.status.cpu().numpy()
    cnt = fw.counters.cpu().numpy()
    ok = st == 0                  # the zones that get gradients
    steps = int(cnt[ok, 0].sum())
    flops = metrics.adjoint_ops(info, steps, K, net.self_heating)
    achieved = flops / (adj_ms * 1e-3) / 1e12
    return {"workload": workload_desc(name, Z) + ", 6 cotangents per zone",
            "value": int(ok.sum()) * K / ((fwd_ms + adj_ms) * 1e-3), "unit": "gradients/s",
            "gradient_length": net.R, "forward_ms": fwd_ms, "reverse_ms": adj_ms,
            "repeats": repeats, "forward_ms_each": fwd, "reverse_ms_each": rev,
            "tape_checkpoint_stride": stride, "tape_max_steps": max_steps,
            "zones_ok": int(ok.sum()),
            "zone_status_counts": {str(k): int(v) for k, v in zip(*np.unique(st, return_counts=True))},
            "forward_launch": fl,
            "reverse_ms_full_tape": full_ms,
            "forward_kernel": "k_burn_coop" if fk == "coop" else "k_burn_persistent",
            "adjoint_kernel": kname,
            "roofline": {"bound": "alu", "kernel": kname,
                         "achieved": achieved,
                         "peak": metrics.FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / metrics.FP64_PEAK_TFLOPS,
                         "traffic": profiled_traffic(kname, Z, None, workload=name),
                         "flops_per_launch": flops,
                         "timed": "CUDA events around nb_burn_adjoint: the claim-order sort "
                                  "and the adjoint kernel, which recomputes every checkpointed "
                                  "block"}}


def multi_bench(nb, torch, dev, flush) -> dict:
    """Several networks in one launch: 16384 zones of the self-heating chain
    and 4096 zones of the 48-species network, all to the chain's t_end,
    burned by one nb_burn_multi launch, against the same two sets burned one
    after the other (each with its own default, autotuned-free launch)."""
    sets = []
    for name, Z in (("chain13_heat", 16384), ("net48", 4096)):
        net, z, s = gen.problem(name, Z)
        sets.append(dict(net=nb.Network(net), Y0=torch.from_numpy(z["Y"]).to(dev),
                         T9=torch.from_numpy(z["T9"]).to(dev),
                         rho=torch.from_numpy(z["rho"]).to(dev)))
    _, _, s0 = gen.problem("chain13_heat", 1)
    te, rt, at = s0["t_end"], s0["rtol"], s0["atol"]
    outs = nb.burn_multi(sets, te, rt, at)                    # warm-up
    for d in sets:
        nb.burn(d["net"], d["Y0"], d["T9"], d["rho"], te, rt, at)
    torch.cuda.synchronize()
    flush.fill_(4.0)
    a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    a.record()
    outs = nb.burn_multi(sets, te, rt, at)
    b.record()
    for d in sets:
        nb.burn(d["net"], d["Y0"], d["T9"], d["rho"], te, rt, at)
    c.record()
    torch.cuda.synchronize()
    multi_ms, seq_ms = a.elapsed_time(b), b.elapsed_time(c)
    Z = sum(int(d["Y0"].shape[0]) for d in sets)
    ok = sum(int((o.status == 0).sum()) for o in outs)
    return {"workload": "13-species self-heating chain (16384 zones) + 48-species network "
                        "(4096 zones), t_end 1e-3 s, rtol 1e-8, atol 1e-12",
            "value": Z / (multi_ms * 1e-3), "unit": "zone-burns/s", "ms": multi_ms,
            "sequential_ms": seq_ms, "zones_ok": ok}


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["native", "reference"], default="native")
    p.add_argument("--workload", default=WORKLOAD, choices=sorted(gen.CONFIGS))
    p.add_argument("--zones", type=int, default=0, help="0: the workload's zone count")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--sample-parity", type=int, default=256,
                   help="check N seeded zones of the timed launch against the oracle")
    p.add_argument("--configs", default="cfg0,cfg2,cfg4",
                   help="comma-separated entries of the configuration table to add")
    p.add_argument("--t-end", type=float, default=None,
                   help="override t_end (profiling of a shorter burn only)")
    p.add_argument("--blocks-per-sm", type=int, default=0)
    p.add_argument("--threads-per-block", type=int, default=0)
    p.add_argument("--ws-in-shared", type=int, default=-1)
    p.add_argument("--specialize", type=int, default=None,
                   help="-1 generic kernel, 0 automatic, 1..3 specialised variant")
    p.add_argument("--kernel", default="persistent", choices=["persistent", "coop"],
                   help="the main workload's kernel (coop: one warp per zone); "
                        "persistent lets the autotuner choose")
    p.add_argument("--warps-per-zone", type=int, default=0,
                   help="with --kernel coop: a block of 2 or 4 warps per zone")
    p.add_argument("--cpu-zones", type=int, default=8192)
    p.add_argument("--ref-zones", type=int, default=4096)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--adjoint", action=argparse.BooleanOptionalAction, default=True)
    p.add_argument("--cfg4-adjoint", action="store_true",
                   help="add the 128-species network's 8192-zone adjoint over all 600 "
                        "multipliers (a few minutes)")
    p.add_argument("--multi", action=argparse.BooleanOptionalAction, default=True)
    args = p.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
