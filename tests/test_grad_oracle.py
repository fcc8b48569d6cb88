"""Pins of the finite-difference reference for the backward (oracle/hef_grad)
against closed forms and exact invariants of Algorithm 1.  CPU only.

 * single hyperedge: R_e = 1/w_e, so dR_e/dw_e = -1/w_e^2 (hand derivation);
 * homogeneity: scaling every weight by c scales W and D by c, so M = D^-1 W,
   the deflation and Q are unchanged while Q_H scales by c: R(c w) = R(w)/c,
   and by Euler's theorem sum_e w_e dL/dw_e = -L for L = sum_e g_e R_e;
 * starts: scaling one chain's start, or adding a trivial eigenvector (the
   constant) to it, leaves the Krylov spans and hence R unchanged."""
import json
import os

import numpy as np
import pytest

from netlists import start_block
from oracle import hef_grad as G
from tests._hypergraphs import from_lists, random_hypergraph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def test_fd_single_hyperedge_closed_form():
    case = json.load(open(GOLDEN))["single_hyperedge"]
    H = from_lists(case["n"], case["edges"], case["w"])
    x0c, x0b = start_block(H.n, H.m, 1, 3)
    g = np.ones(H.m)
    vals, valid = G.weight_gradient(H.n, H.eptr, H.pins, H.w, x0c, x0b, 2, g, [0])
    assert valid.all()
    assert abs(vals[0] - case["dR_dw"][0]) < 1e-8
    d, ok = G.directional(H.n, H.eptr, H.pins, H.w, x0c, x0b, 2, g, np.zeros(H.m),
                          np.ones_like(x0c), np.ones_like(x0b), h=1e-3)
    assert ok and abs(d) < 1e-9


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fd_euler_homogeneity(seed):
    H = random_hypergraph(30, 25, 6, seed, weights=True)
    x0c, x0b = start_block(H.n, H.m, 2, seed)
    k = 3
    g = np.random.default_rng(seed).uniform(0.5, 1.5, H.m)
    L, _ = G.loss(H.n, H.eptr, H.pins, H.w, x0c, x0b, k, g)
    # every coordinate separately (pins the per-coordinate indexing and step)
    vals, valid = G.weight_gradient(H.n, H.eptr, H.pins, H.w, x0c, x0b, k, g, range(H.m))
    assert valid.all()
    assert abs((H.w * vals).sum() + L) < 1e-7 * L
    # along w itself
    d, ok = G.directional(H.n, H.eptr, H.pins, H.w, x0c, x0b, k, g, H.w)
    assert ok and abs(d + L) < 1e-7 * L


@pytest.mark.parametrize("seed", [0, 1])
def test_fd_start_invariances(seed):
    H = random_hypergraph(30, 25, 6, seed, weights=True)
    x0c, x0b = start_block(H.n, H.m, 2, seed)
    k = 3
    g = np.random.default_rng(seed).uniform(0.5, 1.5, H.m)
    L, _ = G.loss(H.n, H.eptr, H.pins, H.w, x0c, x0b, k, g)
    zero_w = np.zeros(H.m)
    one_chain = x0c * np.array([1.0, 0.0])          # scale clique start 0
    d1, ok1 = G.directional(H.n, H.eptr, H.pins, H.w, x0c, x0b, k, g, zero_w, one_chain, None)
    const = np.ones_like(x0c)                       # constant on the clique starts
    d2, ok2 = G.directional(H.n, H.eptr, H.pins, H.w, x0c, x0b, k, g, zero_w, const, None)
    assert ok1 and ok2
    assert abs(d1) < 1e-7 * L and abs(d2) < 1e-7 * L
    # a generic direction does move L (the test above is not vacuous)
    rnd = np.random.default_rng(seed + 10).standard_normal(x0c.shape)
    d3, _ = G.directional(H.n, H.eptr, H.pins, H.w, x0c, x0b, k, g, zero_w, rnd, None)
    assert abs(d3) > 1e-4 * L
