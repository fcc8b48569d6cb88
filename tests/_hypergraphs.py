"""Small hand-built hypergraphs used by several test files (inputs only)."""
import numpy as np

from netlists import Netlist


def from_lists(n, edges, w=None):
    eptr = np.zeros(len(edges) + 1, dtype=np.int64)
    eptr[1:] = np.cumsum([len(e) for e in edges])
    pins = np.array([p for e in edges for p in e], dtype=np.int32)
    if w is None:
        w = np.ones(len(edges))
    return Netlist(n=n, eptr=eptr, pins=pins, w=np.asarray(w, dtype=np.float64))


def random_hypergraph(n, m, max_size, seed, weights=False, min_size=2):
    rng = np.random.default_rng(seed)
    edges = []
    for _ in range(m):
        k = int(rng.integers(min_size, max_size + 1))
        edges.append(list(rng.choice(n, size=min(k, n), replace=False)))
    w = rng.uniform(0.5, 2.0, size=m) if weights else None
    return from_lists(n, edges, w)


def random_graph(n, m, seed, weights=True, connected=True):
    """Random 2-pin hypergraph; with ``connected`` a spanning path is added."""
    rng = np.random.default_rng(seed)
    edges = set()
    if connected:
        perm = rng.permutation(n)
        for i in range(n - 1):
            a, b = int(perm[i]), int(perm[i + 1])
            edges.add((min(a, b), max(a, b)))
    while len(edges) < m:
        a, b = rng.choice(n, size=2, replace=False)
        edges.add((int(min(a, b)), int(max(a, b))))
    edges = sorted(edges)
    w = rng.uniform(0.5, 2.0, size=len(edges)) if weights else None
    return from_lists(n, [list(e) for e in edges], w)
