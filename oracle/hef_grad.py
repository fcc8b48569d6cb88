"""Finite-difference derivatives of the FP64 oracle's hyperedge resistances
(Algorithm 1, Eq. R), the reference for the backward of the CUDA path.

TEST INFRASTRUCTURE ONLY: imported by the tests; the GPU path never imports
it.  The paper defines only the forward.  The derivative checked here is the
one of L = sum_e g_e R_e(w, x0) for a fixed weighting g, where R comes from
``hef_oracle.hyperedge_resistance``: R_e is piecewise smooth (the max over
basis columns in Eq. R and the arg-max/arg-min pins of Eq. ratios switch on
ties), so a difference quotient only means the derivative when the routing
(argvec, pmax, pmin) is the same at both ends of the step; each function
reports whether it was.

Central differences, (L(u + h d) - L(u - h d)) / (2 h): truncation error
O(h^2) times the third derivative, rounding error about eps * |L| / h.
"""
from __future__ import annotations

import numpy as np

from . import hef_oracle as O


def _forward(n, eptr, pins, w, x0_c, x0_b, k, clique):
    return O.hyperedge_resistance(n, eptr, pins, w, x0_c, x0_b, k, clique)


def _routing(out):
    return (np.asarray(out["argvec"]), np.asarray(out["pmax"]), np.asarray(out["pmin"]))


def _same_routing(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def loss(n, eptr, pins, w, x0_c, x0_b, k, g, clique="hyperedge"):
    """L = sum_e g_e R_e and the oracle's forward output."""
    out = _forward(n, eptr, pins, w, x0_c, x0_b, k, clique)
    return float(np.dot(g, out["R"])), out


def directional(n, eptr, pins, w, x0_c, x0_b, k, g, dw, dx0_c=None, dx0_b=None, h=1e-6,
                clique="hyperedge"):
    """Central difference of L along (dw, dx0_c, dx0_b) with step h (the
    direction is used as given, so h is relative to its scale).
    Returns (derivative, routing unchanged between the two ends)."""
    w = np.asarray(w, dtype=np.float64)
    zc = np.zeros_like(x0_c) if dx0_c is None else dx0_c
    zb = np.zeros_like(x0_b) if dx0_b is None else dx0_b
    Lp, op = loss(n, eptr, pins, w + h * dw, x0_c + h * zc, x0_b + h * zb, k, g, clique)
    Lm, om = loss(n, eptr, pins, w - h * dw, x0_c - h * zc, x0_b - h * zb, k, g, clique)
    return (Lp - Lm) / (2.0 * h), _same_routing(_routing(op), _routing(om))


def weight_gradient(n, eptr, pins, w, x0_c, x0_b, k, g, coords, rel_h=1e-6,
                    clique="hyperedge"):
    """dL/dw_e for e in coords by central differences with h = rel_h * w_e.
    Returns (values, valid) where valid[i] says the routing of every hyperedge
    was the same at w_e - h and w_e + h."""
    w = np.asarray(w, dtype=np.float64)
    vals = np.zeros(len(coords))
    valid = np.zeros(len(coords), dtype=bool)
    for i, e in enumerate(coords):
        h = rel_h * w[e]
        d = np.zeros_like(w)
        d[e] = 1.0
        vals[i], valid[i] = directional(n, eptr, pins, w, x0_c, x0_b, k, g, d, h=h, clique=clique)
    return vals, valid
