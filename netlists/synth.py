"""Seeded generators for netlist-shaped hypergraphs on a 2-D placement grid.

The paper evaluates on the ISPD98 and Titan23 VLSI netlists (Section IV),
which are not shipped here.  These generators stand in for them with the
shapes of those benchmarks: cells on a grid (node id = y * nx + x), nets
(hyperedges) with a heavy majority of 2-3 pin nets and a long tail, pins drawn
from a neighbourhood of a random anchor cell, and optionally a small share of
long-range pins.

Everything here is plain numpy driven by ``numpy.random.default_rng(seed)``;
nothing computes expansions, Krylov vectors or resistances.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Netlist:
    """A hypergraph H = (V, E, w) in edge-major (CSC) incidence form.

    ``eptr[m+1]`` (int64) delimits each hyperedge's pins in ``pins[P]``
    (int32 node ids, distinct within a hyperedge); ``w[m]`` are the positive
    hyperedge weights (float64).
    """

    n: int
    eptr: np.ndarray
    pins: np.ndarray
    w: np.ndarray
    nx: int = 0
    ny: int = 0
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.eptr.shape[0] - 1)

    @property
    def P(self) -> int:
        return int(self.eptr[-1])

    def sizes(self) -> np.ndarray:
        return np.diff(self.eptr)


# ----------------------------------------------------------------------------
# pin-count laws


def _sizes_geometric(rng, m, cap):
    """2 + Geometric(p=0.5) on {0,1,...} (mean 3), capped at ``cap``."""
    g = rng.geometric(0.5, size=m) - 1  # numpy's geometric starts at 1
    return np.minimum(2 + g, cap).astype(np.int64)


def _sizes_pareto_tail(rng, m, cap, alpha=2.2, xm=4.0):
    """2 or 3 pins with probability 0.4 each; otherwise a Pareto(alpha) tail
    min(cap, ceil(xm * U^(-1/alpha)))."""
    u = rng.random(m)
    sizes = np.where(u < 0.4, 2, 3).astype(np.int64)
    tail = u >= 0.8
    ut = rng.random(int(tail.sum()))
    ut = np.maximum(ut, np.finfo(np.float64).tiny)
    sizes[tail] = np.minimum(cap, np.ceil(xm * ut ** (-1.0 / alpha))).astype(np.int64)
    return sizes


# ----------------------------------------------------------------------------
# pin placement


def _place_pins(rng, nx, ny, anchors, sizes, radius):
    """For each hyperedge, the anchor cell plus ``size-1`` distinct other cells
    drawn uniformly without replacement from the Chebyshev box of ``radius``
    around the anchor, clipped to the grid.  Returns a list (one array per
    hyperedge) in generation order."""
    m = anchors.shape[0]
    out = [None] * m
    ax = anchors % nx
    ay = anchors // nx
    for r in np.unique(radius):
        idx = np.nonzero(radius == r)[0]
        d = np.arange(-r, r + 1)
        ox, oy = np.meshgrid(d, d, indexing="xy")
        ox = ox.ravel()
        oy = oy.ravel()
        keep = ~((ox == 0) & (oy == 0))
        ox = ox[keep]
        oy = oy[keep]
        # process in chunks to bound memory
        chunk = max(1, (1 << 24) // ox.size)
        for c0 in range(0, idx.size, chunk):
            sel = idx[c0:c0 + chunk]
            cx = ax[sel, None] + ox[None, :]
            cy = ay[sel, None] + oy[None, :]
            valid = (cx >= 0) & (cx < nx) & (cy >= 0) & (cy < ny)
            keys = rng.random(cx.shape, dtype=np.float32)
            keys[~valid] = 2.0
            order = np.argsort(keys, axis=1, kind="stable")
            cell = cy * nx + cx
            ranked = np.take_along_axis(cell, order, axis=1)
            ranked_ok = np.take_along_axis(valid, order, axis=1)
            for t, e in enumerate(sel):
                s = int(sizes[e]) - 1
                if s > 0 and not ranked_ok[t, s - 1]:
                    raise ValueError("neighbourhood too small for hyperedge size")
                out[e] = np.concatenate(([anchors[e]], ranked[t, :s]))
    return out


def _long_range(rng, n, pin_lists, p):
    """Replace each non-anchor pin, with probability p, by a uniform random
    node not already in the hyperedge."""
    if p <= 0:
        return pin_lists
    for e, pl in enumerate(pin_lists):
        if pl.size < 2:
            continue
        hit = np.nonzero(rng.random(pl.size - 1) < p)[0] + 1
        for t in hit:
            while True:
                v = int(rng.integers(0, n))
                if v not in pl:
                    pl[t] = v
                    break
    return pin_lists


def grid_netlist(nx, ny, m, seed, size_law="geometric16", radius_law="fixed3",
                 long_range=0.0, weight_law="unit", name=""):
    """Generate a netlist-shaped hypergraph on an ``nx`` x ``ny`` grid.

    size_law: ``geometric16`` (2 + Geometric(0.5), cap 16) or ``pareto400``
    (80 % 2-3 pins, Pareto(2.2) tail capped at 400).
    radius_law: ``fixed3`` (Chebyshev radius 3) or ``sqrt`` (radius
    max(3, ceil(sqrt(|e|)))).
    weight_law: ``unit`` or ``loguniform`` (exp U(ln 0.5, ln 2)).
    """
    rng = np.random.default_rng(seed)
    n = nx * ny
    if size_law == "geometric16":
        sizes = _sizes_geometric(rng, m, 16)
    elif size_law == "pareto400":
        sizes = _sizes_pareto_tail(rng, m, 400)
    else:
        raise ValueError(size_law)
    if radius_law == "fixed3":
        radius = np.full(m, 3, dtype=np.int64)
    elif radius_law == "sqrt":
        radius = np.maximum(3, np.ceil(np.sqrt(sizes)).astype(np.int64))
    else:
        raise ValueError(radius_law)
    anchors = rng.integers(0, n, size=m)
    pin_lists = _place_pins(rng, nx, ny, anchors, sizes, radius)
    pin_lists = _long_range(rng, n, pin_lists, long_range)
    eptr = np.zeros(m + 1, dtype=np.int64)
    eptr[1:] = np.cumsum(sizes)
    pins = np.concatenate(pin_lists).astype(np.int32)
    if weight_law == "unit":
        w = np.ones(m, dtype=np.float64)
    elif weight_law == "loguniform":
        w = np.exp(rng.uniform(math.log(0.5), math.log(2.0), size=m))
    else:
        raise ValueError(weight_law)
    return Netlist(n=n, eptr=eptr, pins=pins, w=w, nx=nx, ny=ny, name=name)


def start_block(n, m, S, seed):
    """Random start vectors for the two expansions: ``x0_c`` (n x S) for the
    clique expansion and ``x0_b`` ((n+m) x S) for the star expansion, i.i.d.
    uniform on (-1, 1), float64, row-major (S contiguous values per row)."""
    rng = np.random.default_rng([seed, 0x5EED])
    x0_c = rng.uniform(-1.0, 1.0, size=(n, S))
    x0_b = rng.uniform(-1.0, 1.0, size=(n + m, S))
    return x0_c, x0_b


def window_subhypergraph(H: Netlist, x0, x1, y0, y1, name=""):
    """Induced sub-hypergraph of the grid window [x0,x1) x [y0,y1): the cells
    inside (renumbered row-major within the window) and the hyperedges whose
    pins all lie inside."""
    nx = H.nx
    cx = np.arange(H.n) % nx
    cy = np.arange(H.n) // nx
    inside = (cx >= x0) & (cx < x1) & (cy >= y0) & (cy < y1)
    newid = np.full(H.n, -1, dtype=np.int64)
    newid[inside] = (cy[inside] - y0) * (x1 - x0) + (cx[inside] - x0)
    sizes = H.sizes()
    edge_of = np.repeat(np.arange(H.m), sizes)
    bad = np.zeros(H.m, dtype=bool)
    np.logical_or.at(bad, edge_of, ~inside[H.pins])
    keep = ~bad
    ks = sizes[keep]
    eptr = np.zeros(int(keep.sum()) + 1, dtype=np.int64)
    eptr[1:] = np.cumsum(ks)
    pins = newid[H.pins[keep[edge_of]]].astype(np.int32)
    return Netlist(n=(x1 - x0) * (y1 - y0), eptr=eptr, pins=pins, w=H.w[keep].copy(),
                   nx=x1 - x0, ny=y1 - y0, name=name)


# ----------------------------------------------------------------------------
# named workloads (sizes of the evaluation configurations)

WORKLOADS = {
    # FP64 small case: 64x32 grid, 2,300 nets, 2+Geom(0.5) pins (cap 16),
    # radius-3 neighbourhoods, unit weights; k=10 per operator, S=1.
    "grid64x32_m2300": dict(nx=64, ny=32, m=2300, seed=0, size_law="geometric16",
                            radius_law="fixed3", long_range=0.0, weight_law="unit",
                            k=10, S=1),
    # IBM18-sized case: 500x420 grid (n=210,000), 200,000 nets, 80 % 2-3
    # pins with a Pareto(2.2) tail capped at 400, 2 % long-range pins.
    "grid500x420_m200k": dict(nx=500, ny=420, m=200000, seed=2, size_law="pareto400",
                              radius_law="sqrt", long_range=0.02, weight_law="unit",
                              k=20, S=4),
    # 1.2M-cell case for the BF16-storage form.
    "grid1200x1000_m1300k": dict(nx=1200, ny=1000, m=1300000, seed=3,
                                 size_law="geometric16", radius_law="fixed3",
                                 long_range=0.0, weight_law="unit", k=24, S=8),
    # differentiation case: log-uniform weights on (0.5, 2).
    "grid500x400_m210k_logw": dict(nx=500, ny=400, m=210000, seed=5,
                                   size_law="geometric16", radius_law="fixed3",
                                   long_range=0.0, weight_law="loguniform", k=10, S=1),
    # FD-sized differentiation case (same law as above at the small size).
    "grid64x32_m2300_logw": dict(nx=64, ny=32, m=2300, seed=0, size_law="geometric16",
                                 radius_law="fixed3", long_range=0.0,
                                 weight_law="loguniform", k=10, S=1),
}


def workload(name):
    """Build a named workload; returns (Netlist, k, S)."""
    cfg = dict(WORKLOADS[name])
    k = cfg.pop("k")
    S = cfg.pop("S")
    return grid_netlist(name=name, **cfg), k, S


def batch_sizes(G=64, seed=4000):
    """Node counts of the batched case: n_g = round(exp U(ln 5e3, ln 1.5e5)),
    m_g = round(1.05 n_g), on near-square grids."""
    rng = np.random.default_rng(seed)
    ns = np.round(np.exp(rng.uniform(math.log(5e3), math.log(1.5e5), size=G))).astype(int)
    out = []
    for g, n in enumerate(ns):
        nx = int(math.ceil(math.sqrt(n)))
        ny = int(math.ceil(n / nx))
        out.append((nx, ny, int(round(1.05 * nx * ny)), seed + g))
    return out
