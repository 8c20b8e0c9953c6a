"""Comparison of GPU burns with the CPU oracle (shared by the GPU tests,
``__graft_entry__.smoke`` and the benchmark's sampled check).

The bar, per zone:
  * status equal; accepted-step counts within 2 of each other;
  * zones whose accepted-step counts agree: every species within
    1e-9 |Y_oracle| + max(1e-5 atol, 1e-15 max_j |Y_oracle,j|), T9 and E
    within 1e-9 relative (+1e-12 absolute for E);
  * zones whose counts differ by 1 or 2 took a different (equally valid)
    step sequence; they must agree to the integration tolerance,
    1e-4 |Y| + atol, and be rare (< 1% of zones).
The method resolves a species only to its weight w = atol + rtol |Y| (the
Newton test stops at 1e-3 w, the error test at w), so species near or below
atol agree between two correct implementations only to a fraction of atol,
hence the 1e-5 atol absolute floor (1e-17 at the workloads' atol = 1e-12).
A species' rate of change is a sum of terms proportional to the zone's large
abundances, so its absolute rounding error follows theirs, not its own size:
the floor is at least a few ulps of the zone's largest abundance,
1e-15 max_j |Y_j| (2.5e-16 when Y_0 = 1/4 dominates).
Networks with tabulated rates take the wider same-step bar TABULATED below.
"""
from __future__ import annotations

import numpy as np


# Networks with tabulated rates: ln lambda is piecewise linear in T9, so the
# right-hand side has kinks at the table's temperatures.  Where a step
# straddles a kink its error estimate, and so the step sizes around it,
# depend sharply on where it lands, and two implementations that differ at
# rounding level agree only to the method's own resolution: each entry to
# its weight w = atol + rtol |Y| (the error test), T9 and E to 1e-6
# relative.  Measured over 2048 zones (host run of the device code against
# the oracle): 0.16 of this bar at most, T9 4e-8, 0.6 % of zones on a
# different step sequence.  Near a kink the error test can accept or reject
# a step on rounding, each flip shifting the step sequence; a zone crosses at
# most the grid's 12 temperatures, so accepted-step counts may differ by up to
# 12 (such zones are still held to the integration tolerance).  Measured on
# the GPU: 3.
TABULATED = dict(same_rel=1e-6, same_w=1.0, scalar_rel=1e-6, max_diverged_frac=0.03,
                 max_step_diff=12)


def compare(gpu: dict, ora: dict, atol: float, max_step_diff: int = 2,
            max_diverged_frac: float = 0.01, same_rel: float = 1e-9, same_w: float = 0.0,
            scalar_rel: float = 1e-9, rtol: float = 1e-8) -> dict:
    Yg, Yo = np.asarray(gpu["Y"]), np.asarray(ora["Y"])
    sg, so = np.asarray(gpu["status"]), np.asarray(ora["status"])
    cg, co = np.asarray(gpu["counters"]), np.asarray(ora["counters"])
    Z = Yo.shape[0]
    report = {"zones": Z}
    bad = np.where(sg != so)[0]
    assert bad.size == 0, f"status differs in zones {bad[:10]}: gpu {sg[bad[:10]]} oracle {so[bad[:10]]}"
    ok = so == 0
    dacc = cg[:, 0].astype(np.int64) - co[:, 0].astype(np.int64)
    report["max_step_diff"] = int(np.abs(dacc[ok]).max()) if ok.any() else 0
    assert report["max_step_diff"] <= max_step_diff, \
        f"accepted steps differ by {report['max_step_diff']}"
    same = ok & (dacc == 0)
    diverged = ok & (dacc != 0)
    report["diverged_zones"] = int(diverged.sum())
    assert diverged.sum() <= max(1, int(max_diverged_frac * Z)), \
        f"{diverged.sum()} of {Z} zones took a different step sequence"
    floor = np.maximum(1e-5 * atol, 1e-15 * np.abs(Yo).max(axis=1, keepdims=True))
    tol = same_rel * np.abs(Yo) + floor + same_w * (atol + rtol * np.abs(Yo))
    err = np.abs(Yg - Yo)
    viol = (err > tol) & same[:, None]
    rel = np.where(np.abs(Yo) > 1e-20, err / np.maximum(np.abs(Yo), 1e-300), 0.0)
    report["max_rel_Y"] = float(rel[same].max()) if same.any() else 0.0
    report["max_abs_small_Y"] = float(np.where(np.abs(Yo) <= 1e-20, err, 0)[same].max()) if same.any() else 0.0
    zi = np.where(viol.any(1))[0]
    assert zi.size == 0, (f"{zi.size} zones exceed the same-step bar, e.g. zone {zi[0]}: "
                          f"gpu {Yg[zi[0]][viol[zi[0]]][:4]} oracle {Yo[zi[0]][viol[zi[0]]][:4]}")
    if diverged.any():
        loose = 1e-4 * np.abs(Yo) + atol
        zl = np.where(((err > loose) & diverged[:, None]).any(1))[0]
        assert zl.size == 0, f"diverged zones {zl[:5]} differ beyond the integration tolerance"
    for key, floor in (("T9", 0.0), ("E", 1e-12)):
        if key in gpu and key in ora and gpu[key] is not None:
            a, b = np.asarray(gpu[key]), np.asarray(ora[key])
            e = np.abs(a - b)
            lim = np.where(same, scalar_rel * np.abs(b) + floor, 1e-4 * np.abs(b) + 1e-8)
            report[f"max_rel_{key}"] = float((e / np.maximum(np.abs(b), 1e-300))[ok].max()) if ok.any() else 0.0
            zb = np.where(ok & (e > lim))[0]
            assert zb.size == 0, f"{key} differs in zones {zb[:5]}: {a[zb[:5]]} vs {b[zb[:5]]}"
    return report


def to_numpy(res) -> dict:
    return {k: getattr(res, k).cpu().numpy() for k in ("Y", "T9", "E", "counters", "status")}
