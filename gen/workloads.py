"""Deterministic synthetic workloads for the batched reaction-network burn.

The paper's own runs (Sec. 3: a Castro 1D He detonation with the pynucastro
He-C-Fe, subch_simple and aprox19 networks) need the JINA ReacLib database,
weak-rate tables, the Helmholtz EOS table and Castro, none of which exist
here.  These seeded stand-ins have the paper's shapes instead: an alpha-chain
of 13 nuclei (the aprox13 shape of the Sec. 2 nuclide list), random networks
of 48 species / 180 rates (the size class of He-C-Fe, 36 isotopes and 149
rates, Sec. 2) and 128 / 600, temperatures spanning the 0.175-3 GK of Sec. 3
and densities up to 1e9 g/cm^3.

Every array is drawn with numpy ``Generator(PCG64(seed))``.  Draw order is
part of the definition and must not change:

* fit coefficients, for R rates, in this order: a0 ~ U[5,20], a1 ~ U[-20,0],
  a2 ~ U[-50,-10], (a3, a4, a5) ~ N(0, 0.5) as one (3, R) draw, a6 ~ U[-1.5,0];
* energy per rate Q ~ U[1,10] where a workload needs it;
* per-zone values come from three child streams of ``SeedSequence(1000+i)``
  (temperature, density, composition), so the first Z' zones of a workload
  are the same whatever Z is drawn; log-uniform means exp(U[ln a, ln b]).

Random networks (A_i = i + 1, so mass number is conserved by construction):
one-body rates split X into a pair with A_p + A_q = A_X; two- and three-body
reactant tuples are sorted, with probability 0.8 one reactant is one of the 4
lightest species; the product is the single species with the summed A when it
exists and a fair coin says so, else a pair with that sum.  Duplicate rates
and identity rates are redrawn.  The whole network is redrawn from seed+1,
seed+2, ... until the species graph is connected.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

# Workload table.  Keys name what the workload is.
CONFIGS = {
    # 13-species alpha chain, fixed T and rho.
    "chain13": dict(kind="chain", literal=False, heat=False, Z=4096,
                    T9=(1.0, 4.0), rho=(1e5, 1e8), t_end=1e-3,
                    rtol=1e-8, atol=1e-12, zone_seed=1000, Q=False),
    # Same species with the literal 13-rate list (adds Y0 + Y0 -> Y1).
    "chain13_literal": dict(kind="chain", literal=True, heat=False, Z=4096,
                            T9=(1.0, 4.0), rho=(1e5, 1e8), t_end=1e-3,
                            rtol=1e-8, atol=1e-12, zone_seed=1000, Q=False),
    # alpha chain with self-heating (T evolves with Y).
    "chain13_heat": dict(kind="chain", literal=False, heat=True, Z=65536,
                         T9=(0.5, 5.0), rho=(1e5, 1e8), t_end=1e-3,
                         rtol=1e-8, atol=1e-12, zone_seed=1001, Q=True),
    # The self-heating chain with its captures on species 1..11 taken as
    # effective (alpha,p)(p,gamma) rates (the aprox-style approximation of
    # the paper's Sec. 2): each such rate combines four fits.  Same zones as
    # chain13_heat.
    "chain13_heat_ap": dict(kind="chain", literal=False, heat=True, Z=65536,
                            T9=(0.5, 5.0), rho=(1e5, 1e8), t_end=1e-3,
                            rtol=1e-8, atol=1e-12, zone_seed=1001, Q=True,
                            ap_from=1),
    # The self-heating chain with weak screening of every rate: charges
    # Z_i = A_i / 2, and a synthetic plasma parameter per zone, zeta ~ U[1, 2]
    # (the chain's initial composition gives 1.5).  Same zones as
    # chain13_heat otherwise.
    "chain13_heat_scr": dict(kind="chain", literal=False, heat=True, Z=65536,
                             T9=(0.5, 5.0), rho=(1e5, 1e8), t_end=1e-3,
                             rtol=1e-8, atol=1e-12, zone_seed=1001, Q=True,
                             screen=True, zeta=(1.0, 2.0)),
    # The self-heating chain with reactions 0..5 (triple-alpha and the first
    # five captures) given as tables (TabularRate,
    # the paper's Sec. 2: rates tabulated in (rho Ye, T)): each table is its
    # fit's ln lambda at the grid's temperatures plus a density slope and
    # noise, on a 5 x 12 grid in (log10 rho Ye, T9); charges Z_i = A_i / 2.
    "chain13_heat_tab": dict(kind="chain", literal=False, heat=True, Z=65536,
                             T9=(0.5, 5.0), rho=(1e5, 1e8), t_end=1e-3,
                             rtol=1e-8, atol=1e-12, zone_seed=1001, Q=True,
                             tab=(0, 6)),
    # Random sparse network, 48 species / 180 rates, fixed T and rho.
    "net48": dict(kind="random", N=48, mix=(60, 100, 20), topo_seed=2,
                  heat=False, Z=262144, T9=(0.3, 6.0), rho=(1e4, 1e9),
                  t_end=1e-2, rtol=1e-8, atol=1e-12, zone_seed=1002, Q=False),
    # Same network, energy per rate drawn, for the sensitivity workload.
    "net48_adjoint": dict(kind="random", N=48, mix=(60, 100, 20), topo_seed=2,
                          heat=False, Z=16384, T9=(0.3, 6.0), rho=(1e4, 1e9),
                          t_end=1e-2, rtol=1e-8, atol=1e-12, zone_seed=1003,
                          Q=True),
    # Large random network, 128 species / 600 rates, self-heating.
    "net128_heat": dict(kind="random", N=128, mix=(200, 333, 67), topo_seed=4,
                        heat=True, Z=131072, T9=(0.3, 8.0), rho=(1e4, 1e9),
                        t_end=1e-1, rtol=1e-8, atol=1e-12, zone_seed=1004,
                        Q=True),
}

ALPHA_CHAIN_A = np.array([4, 12, 16, 20, 24, 28, 32, 36, 40, 44, 48, 52, 56],
                         dtype=np.float64)


@dataclass
class NetworkSpec:
    name: str
    N: int
    R: int
    reactants: np.ndarray          # int16 [R, 3], -1 padded, sorted
    products: np.ndarray           # int16 [R, 3], -1 padded, sorted
    A: np.ndarray                  # float64 [N] mass numbers
    coeffs: np.ndarray             # float64 [R, 7]
    Q: Optional[np.ndarray] = None  # float64 [R] energy per rate, or None
    scale: Optional[np.ndarray] = None  # float64 [R] constant factor, or None
    self_heating: bool = False
    seed_used: int = 0
    # (alpha,p)(p,gamma) effective rates: ap_pg [R] int8 (1 = effective),
    # ap_coeffs [R, 3, 7] fits of the (a,p), (p,g) and (p,a) channels
    ap_pg: Optional[np.ndarray] = None
    ap_coeffs: Optional[np.ndarray] = None
    # weak-screening strength per reaction, s_r = 0.188 sum Z_a Z_b over the
    # reactants' successive pairs, or None
    screen: Optional[np.ndarray] = None
    # tabulated rates: tab_of [R] (table of reaction r, -1 = its fit), the
    # grid tab_dens [nd] (log10 rho Ye) x tab_t9 [nt], tab_lnl [n_tab, nd, nt]
    # (ln lambda at the nodes), charge [N] (Ye = sum Z_i Y_i)
    tab_of: Optional[np.ndarray] = None
    tab_dens: Optional[np.ndarray] = None
    tab_t9: Optional[np.ndarray] = None
    tab_lnl: Optional[np.ndarray] = None
    charge: Optional[np.ndarray] = None
    extra: dict = field(default_factory=dict)


def _draw_coeffs(rng: np.random.Generator, R: int) -> np.ndarray:
    a0 = rng.uniform(5.0, 20.0, R)
    a1 = rng.uniform(-20.0, 0.0, R)
    a2 = rng.uniform(-50.0, -10.0, R)
    a345 = rng.normal(0.0, 0.5, (3, R))
    a6 = rng.uniform(-1.5, 0.0, R)
    c = np.empty((R, 7), dtype=np.float64)
    c[:, 0], c[:, 1], c[:, 2] = a0, a1, a2
    c[:, 3:6] = a345.T
    c[:, 6] = a6
    return c


def _screen_strengths(reac: np.ndarray, charge: np.ndarray) -> np.ndarray:
    """s_r = 0.188 (Z_1 Z_2 + (Z_1 + Z_2) Z_3 + ...): the weak-screening
    coefficient of each reaction, the reactants taken as successive pairs
    (a capture on the compound of the ones before).  One-body: 0."""
    out = np.zeros(reac.shape[0])
    for r in range(reac.shape[0]):
        zs = [charge[int(v)] for v in reac[r] if v >= 0]
        acc, zsum = 0.0, zs[0]
        for zb in zs[1:]:
            acc += zsum * zb
            zsum += zb
        out[r] = 0.188 * acc
    return out


TAB_DENS = np.array([4.0, 5.0, 6.0, 7.0, 8.0])                  # log10(rho Ye)
TAB_T9 = np.array([0.3, 0.5, 0.7, 1.0, 1.5, 2.0, 3.0, 4.0, 5.0, 6.0, 8.0, 10.0])


def _tables(coeffs: np.ndarray, rows, R: int) -> dict:
    """Synthetic rate tables for reactions ``rows``: the fit's exponent at
    each grid temperature, plus 0.25 (log10 rho Ye - 6) and N(0, 0.1) noise
    per node (its own seed)."""
    rng = np.random.Generator(np.random.PCG64(6))
    rows = list(rows)
    tab_of = np.full(R, -1, dtype=np.int32)
    lnl = np.empty((len(rows), TAB_DENS.size, TAB_T9.size))
    T = TAB_T9
    phi = np.stack([np.ones_like(T), 1 / T, T ** (-1 / 3), T ** (1 / 3), T, T ** (5 / 3),
                    np.log(T)])
    for m, r in enumerate(rows):
        tab_of[r] = m
        base = coeffs[r] @ phi
        lnl[m] = (base[None, :] + 0.25 * (TAB_DENS[:, None] - 6.0)
                  + rng.normal(0.0, 0.1, (TAB_DENS.size, T.size)))
    return dict(tab_of=tab_of, tab_dens=TAB_DENS.copy(), tab_t9=TAB_T9.copy(), tab_lnl=lnl)


def _pad3(t):
    out = [-1, -1, -1]
    for i, v in enumerate(sorted(t)):
        out[i] = int(v)
    return out


def _chain(literal: bool):
    reac, prod = [], []
    reac.append(_pad3((0, 0, 0)))
    prod.append(_pad3((1,)))
    first = 0 if literal else 1
    for i in range(first, 12):
        reac.append(_pad3((i, 0)))
        prod.append(_pad3((i + 1,)))
    return np.array(reac, dtype=np.int16), np.array(prod, dtype=np.int16)


def _connected(N: int, reac: np.ndarray, prod: np.ndarray) -> bool:
    parent = list(range(N))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for r in range(reac.shape[0]):
        members = [int(v) for v in reac[r] if v >= 0] + \
                  [int(v) for v in prod[r] if v >= 0]
        for m in members[1:]:
            ra, rb = find(members[0]), find(m)
            if ra != rb:
                parent[ra] = rb
    root = find(0)
    return all(find(i) == root for i in range(N))


def _random_topology(rng: np.random.Generator, N: int, mix):
    n1, n2, n3 = mix
    seen = set()
    reac, prod = [], []

    def products_for(total_a):
        # single product with index total_a - 1, or a pair (c, d) with
        # (c + 1) + (d + 1) = total_a
        single_ok = total_a - 1 <= N - 1
        if single_ok and rng.random() < 0.5:
            return (total_a - 1,)
        lo = max(0, total_a - N - 1)
        hi = min(total_a - 2, N - 1)
        if lo > hi:
            return None
        c = int(rng.integers(lo, hi + 1))
        d = total_a - c - 2
        if d < 0 or d > N - 1:
            return None
        return tuple(sorted((c, d)))

    def add(rt, pt):
        key = (tuple(sorted(rt)), tuple(sorted(pt)))
        if key[0] == key[1] or key in seen:
            return False
        seen.add(key)
        reac.append(_pad3(rt))
        prod.append(_pad3(pt))
        return True

    count = 0
    while count < n1:
        x = int(rng.integers(1, N))
        a = int(rng.integers(0, x))        # A_p = a + 1 in [1, A_x - 1]
        q = x - a - 1
        if add((x,), tuple(sorted((a, q)))):
            count += 1
    for nbody, target in ((2, n2), (3, n3)):
        count = 0
        while count < target:
            if rng.random() < 0.8:
                rt = [int(rng.integers(0, 4))] + \
                     [int(v) for v in rng.integers(0, N, nbody - 1)]
            else:
                rt = [int(v) for v in rng.integers(0, N, nbody)]
            rt = tuple(sorted(rt))
            total_a = sum(v + 1 for v in rt)
            pt = products_for(total_a)
            if pt is None:
                continue
            if add(rt, pt):
                count += 1
    return np.array(reac, dtype=np.int16), np.array(prod, dtype=np.int16)


def network(name: str) -> NetworkSpec:
    """The reaction network of workload ``name`` (topology + coefficients)."""
    cfg = CONFIGS[name]
    if cfg["kind"] == "chain":
        reac, prod = _chain(cfg["literal"])
        R = reac.shape[0]
        coeffs = _draw_coeffs(np.random.Generator(np.random.PCG64(0)), R)
        Q = None
        if cfg["Q"]:
            Q = np.random.Generator(np.random.PCG64(1)).uniform(1.0, 10.0, R)
        ap_pg = ap_coeffs = None
        if cfg.get("ap_from") is not None:
            # reaction r (r >= 1) captures an alpha on species r
            ap_pg = np.zeros(R, dtype=np.int8)
            ap_pg[cfg["ap_from"]:] = 1
            rng = np.random.Generator(np.random.PCG64(5))
            ap_coeffs = np.zeros((R, 3, 7), dtype=np.float64)
            for c, shift in enumerate((0.0, 4.0, 0.0)):   # (a,p), (p,g), (p,a)
                f = _draw_coeffs(rng, R)
                f[:, 0] += shift            # proton capture faster than (a,p)
                ap_coeffs[:, c, :] = f
        screen = None
        if cfg.get("screen"):
            screen = _screen_strengths(reac, ALPHA_CHAIN_A / 2.0)
        tab = {}
        if cfg.get("tab") is not None:
            tab = _tables(coeffs, range(*cfg["tab"]), R)
            tab["charge"] = ALPHA_CHAIN_A / 2.0
        return NetworkSpec(name=name, N=13, R=R, reactants=reac, products=prod,
                           A=ALPHA_CHAIN_A.copy(), coeffs=coeffs, Q=Q,
                           self_heating=cfg["heat"], seed_used=0,
                           ap_pg=ap_pg, ap_coeffs=ap_coeffs, screen=screen, **tab)
    N = cfg["N"]
    seed = cfg["topo_seed"]
    while True:
        rng = np.random.Generator(np.random.PCG64(seed))
        reac, prod = _random_topology(rng, N, cfg["mix"])
        if _connected(N, reac, prod):
            break
        seed += 1
    R = reac.shape[0]
    coeffs = _draw_coeffs(rng, R)
    Q = rng.uniform(1.0, 10.0, R)
    return NetworkSpec(name=name, N=N, R=R, reactants=reac, products=prod,
                       A=np.arange(1, N + 1, dtype=np.float64), coeffs=coeffs,
                       Q=Q if cfg["Q"] else None, self_heating=cfg["heat"],
                       seed_used=seed)


def zones(name: str, Z: Optional[int] = None) -> dict:
    """Per-zone initial state of workload ``name``: T9 [Z], rho [Z], Y [Z, N].

    The first Z' zones do not depend on Z (prefix-stable draws)."""
    cfg = CONFIGS[name]
    Z = cfg["Z"] if Z is None else int(Z)
    s_t, s_r, s_y = np.random.SeedSequence(cfg["zone_seed"]).spawn(3)
    lo, hi = cfg["T9"]
    T9 = np.exp(np.random.Generator(np.random.PCG64(s_t)).uniform(
        np.log(lo), np.log(hi), Z))
    lo, hi = cfg["rho"]
    rho = np.exp(np.random.Generator(np.random.PCG64(s_r)).uniform(
        np.log(lo), np.log(hi), Z))
    if cfg["kind"] == "chain":
        Y = np.zeros((Z, 13), dtype=np.float64)
        Y[:, 0] = 0.25
    else:
        N = cfg["N"]
        X = np.random.Generator(np.random.PCG64(s_y)).dirichlet(
            [0.3, 0.3, 0.3, 0.3], Z)
        X = X / X.sum(axis=1, keepdims=True)
        Y = np.zeros((Z, N), dtype=np.float64)
        Y[:, :4] = X / np.arange(1, 5, dtype=np.float64)[None, :]
    out = dict(T9=np.ascontiguousarray(T9), rho=np.ascontiguousarray(rho),
               Y=np.ascontiguousarray(Y))
    if cfg.get("zeta") is not None:
        # a fourth child stream: the first three stay those of the other keys
        s_z = np.random.SeedSequence(cfg["zone_seed"]).spawn(4)[3]
        lo, hi = cfg["zeta"]
        out["zeta"] = np.ascontiguousarray(
            np.random.Generator(np.random.PCG64(s_z)).uniform(lo, hi, Z))
    return out


def problem(name: str, Z: Optional[int] = None):
    """(network, zones, settings) of a workload."""
    cfg = CONFIGS[name]
    return network(name), zones(name, Z), dict(
        t_end=cfg["t_end"], rtol=cfg["rtol"], atol=cfg["atol"])


def largest_species(Y: np.ndarray, k: int = 5) -> np.ndarray:
    """Indices [Z, k] of the k largest entries of each row, ties to the
    lower index (the cotangent recipe for the sensitivity workload)."""
    Z, N = Y.shape
    order = np.lexsort((np.broadcast_to(np.arange(N), (Z, N)), -Y), axis=1)
    return np.ascontiguousarray(order[:, :k].astype(np.int64))
