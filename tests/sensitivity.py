"""The adjoint's bar, shared by the GPU tests and the CPU test of the host
build: a gradient computed by the library against the oracle's forward
sensitivity of the same discrete map, along the same recorded trajectory.
Both differentiate one map, so they differ only in rounding: every entry
must lie within 1e-10 of its own size plus SPREAD_FACTOR times the largest
difference the oracle's 15 rounding variants show on that entry (entries far
below the others of their vector, and the gradients of species far below
atol, are where that spread is larger than 1e-10).  The library differs from
the oracle in more rounding sources at once than any variant (elimination
order, summation order, exp): measured with the host build of the library's
adjoint over the five sensitivity workloads, its deviation reached 2.3 times
the variants' largest, on one gradient the variants themselves spread by
1e-8 relative; the factor is 4.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import gen
import oracle

# rounding variants of the sensitivity computation: every combination of the
# summation order, the reversed and the permuted LU order and one-ulp
# transcendentals (the step-size variant does not touch a frozen schedule)
SENS_VARIANTS = tuple(v for v in range(1, 32) if not v & 8)
SPREAD_FACTOR = 4.0



def cotangents(net, Yf, Z):
    """E and the 5 largest final abundances of each zone (one-hot)."""
    top = gen.largest_species(Yf, 5)
    K = 6
    gY = np.zeros((K, Z, net.N))
    gE = np.zeros((K, Z))
    gE[0] = 1.0
    for q in range(5):
        gY[q + 1, np.arange(Z), top[:, q]] = 1.0
    return gY, gE


def oracle_sensitivities(net, z, read, zones, ln_mult=None):
    """Per zone: the oracle's forward sensitivity (dx, dE) along a recorded
    trajectory (read(i) -> dict t, h, k, x of zone i), for the plain oracle
    and each rounding variant."""
    def one(i):
        rec = read(i)
        assert np.isfinite(rec["x"]).all()
        zeta = float(z["zeta"][i]) if "zeta" in z else 0.0
        lm = None if ln_mult is None else (ln_mult[i] if np.ndim(ln_mult) == 2 else ln_mult)
        return [oracle.forward_sensitivity(net, z["T9"][i], z["rho"][i], rec["t"], rec["k"],
                                           rec["x"], ln_mult=lm, zeta=zeta, h=rec["h"],
                                           variant=v) for v in (0,) + SENS_VARIANTS]
    with ThreadPoolExecutor(16) as ex:
        return list(ex.map(one, zones))


def check_entries(got, runs, what):
    """|got - plain| <= 1e-10 |plain| + SPREAD_FACTOR x max over variants
    |variant - plain| + the FP64 resolution of the vector (2^-52 times its
    largest entry: an entry 60 orders below the others, as some rate
    gradients of a stiff zone are, carries no relative precision)."""
    e0 = runs[0]
    spread = np.max([np.abs(v - e0) for v in runs[1:]], axis=0)
    err = np.abs(got - e0)
    # 1e-290: near and below the smallest normal double, where FP64 itself
    # loses relative precision
    resolution = 2.0 ** -52 * np.abs(e0).max()
    bad = err > 1e-10 * np.abs(e0) + SPREAD_FACTOR * spread + resolution + 1e-290
    assert not bad.any(), (what, np.where(bad)[0][:5], got[bad][:3], e0[bad][:3], spread[bad][:3])
    lit = err > 1e-10 * np.abs(e0)
    return int(lit.sum()), int(err.size)


def check_zone(net, gY, gE, gT9, out, sens, i):
    N, R = net.N, net.R
    lit = tot = 0
    for q in range(gY.shape[0]):
        w = gY[q, i]
        ge = gE[q, i] if gE is not None else 0.0
        gt = gT9[q, i] if gT9 is not None else 0.0
        lin = lambda dx, dE, cols: (w @ dx[:N, cols] + ge * dE[cols] +
                                    (gt * dx[N, cols] if net.self_heating else 0.0))
        for name, got, cols in (("d_ln_mult", out["dl"][q, i], slice(0, R)),
                                ("dY0", out["dY0"][q, i], slice(R, R + N)),
                                ("dT0", np.atleast_1d(out["dT0"][q, i]), slice(R + N, R + N + 1))):
            runs = [np.atleast_1d(lin(dx, dE, cols)) for dx, dE in sens[i]]
            a, b = check_entries(got, runs, (i, q, name))
            lit += a
            tot += b
    return lit, tot


