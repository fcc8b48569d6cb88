"""Pins of the downstream oracle (oracle/hef_downstream.py): one coarsening
level of Algorithm 2 (Section III-B) after Algorithm 1 step 6 and Eq.
R_W_update (Section III-A.3).

The paper prints no worked example for these steps, so the oracle is pinned
by (a) hand-derived cases (tests/golden/downstream.json), (b) a library
routine for the sort, (c) an independent, differently structured
formulation of the greedy contraction (the round-based fixed point that
parallel greedy algorithms use), of the local clustering (vectorised over
all seed/cluster pairs) and of the coarsening (set algebra), and (d) the
defining properties of each step on random hypergraphs."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import hef_downstream as D
from tests._hypergraphs import random_hypergraph

GOLD = os.path.join(os.path.dirname(__file__), "golden", "downstream.json")


def _cases():
    return json.load(open(GOLD))["cases"]


def _exact(pairs):
    return [None if p is None else float(Fraction(p[0], p[1])) for p in pairs]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_golden_levels(case):
    n = case["n"]
    eptr = np.array(case["eptr"], dtype=np.int64)
    pins = np.array(case["pins"], dtype=np.int32)
    R = np.array(case["R"], dtype=np.float64)
    eta = np.array(case["eta"], dtype=np.float64)
    ex = case["expect"]
    Ru = D.update_resistance(eptr, pins, R, eta)
    if "R_upd" in ex:
        assert np.allclose(Ru, ex["R_upd"], rtol=1e-15, atol=0)
    order = D.sort_order(Ru)
    assert order.tolist() == ex["order"]
    delta = case.get("delta")
    if delta is None:
        delta = D.quantile_threshold(Ru, np.diff(eptr), case["q"])
        assert delta == ex["delta"]
    owner, contracted = D.contract(n, eptr, pins, order, Ru, delta)
    assert np.flatnonzero(contracted).tolist() == ex["contracted"]
    cluster, nc, eta_next, formed_by = D.clusters(n, eptr, pins, owner, contracted, Ru, eta)
    assert cluster.tolist() == ex["cluster"] and nc == ex["nc"]
    want_eta = ex.get("eta_next") or _exact(ex["eta_next_exact"])
    assert np.allclose(eta_next, want_eta, rtol=1e-15, atol=0)
    if "Q" not in case:
        return
    out = D.level(n, eptr, pins, np.array(case["w"], dtype=np.float64), R,
                  np.array(case["Q"]), np.array(case["QH"]), eta, q=case["q"])
    assert out["target"].tolist() == ex["target"]
    for p, want in enumerate(_exact(ex["dist_exact"])):
        if want is not None:
            assert math.isclose(out["dist"][p], want, rel_tol=1e-15)
    assert out["final"].tolist() == ex["final"] and out["nf"] == ex["nf"]
    assert np.allclose(out["eta"], _exact(ex["eta_final_exact"]), rtol=1e-15, atol=0)
    assert out["eptr"].tolist() == ex["coarse_eptr"]
    assert out["pins"].tolist() == ex["coarse_pins"]
    assert out["w"].tolist() == ex["coarse_w"]
    assert out["emap"].tolist() == ex["emap"]


def _random_level_inputs(seed, n=60, m=90, kmax=6, K=5, ties=False):
    rng = np.random.default_rng(seed)
    H = random_hypergraph(n, m, kmax, seed)
    if ties:  # few distinct values: ties in the sort and at delta
        R = rng.integers(0, 4, size=H.m).astype(np.float64) / 4
    else:
        R = rng.uniform(0, 1, size=H.m)
    eta = rng.uniform(0, 0.5, size=H.n) * (rng.uniform(size=H.n) < 0.5)
    Q = rng.standard_normal((H.n, K))
    QH = rng.uniform(0.5, 2.0, size=K)
    return H, R, eta, Q, QH


@pytest.mark.parametrize("seed", range(6))
def test_sort_matches_lexsort(seed):
    H, R, eta, _, _ = _random_level_inputs(seed, ties=seed % 2 == 0)
    Ru = D.update_resistance(H.eptr, H.pins, R, eta)
    want = np.lexsort((np.arange(H.m), Ru))
    assert D.sort_order(Ru).tolist() == want.tolist()


def test_update_resistance_properties():
    H, R, eta, _, _ = _random_level_inputs(3)
    assert np.array_equal(D.update_resistance(H.eptr, H.pins, R, np.zeros(H.n)), R)
    Ru = D.update_resistance(H.eptr, H.pins, R, eta)
    for e in range(H.m):
        ps = H.pins[H.eptr[e]:H.eptr[e + 1]]
        assert math.isclose(Ru[e], eta[ps].sum() + R[e], rel_tol=1e-13, abs_tol=1e-15)


def _greedy_rounds(n, eptr, pins, rank, cand):
    """The contraction as a fixed point of rounds: in each round a live
    candidate joins if it has the smallest rank among live candidates at all
    of its pins, and a live candidate leaves once a pin is taken."""
    m = len(eptr) - 1
    state = np.where(cand, 0, 2)  # 0 live, 1 in, 2 out
    taken = np.zeros(n, dtype=bool)
    while (state == 0).any():
        best = np.full(n, np.iinfo(np.int64).max)
        for e in np.flatnonzero(state == 0):
            ps = pins[eptr[e]:eptr[e + 1]]
            best[ps] = np.minimum(best[ps], rank[e])
        joins = [e for e in np.flatnonzero(state == 0)
                 if (best[pins[eptr[e]:eptr[e + 1]]] == rank[e]).all()]
        for e in joins:
            state[e] = 1
            taken[pins[eptr[e]:eptr[e + 1]]] = True
        for e in np.flatnonzero(state == 0):
            if taken[pins[eptr[e]:eptr[e + 1]]].any():
                state[e] = 2
    return state == 1


@pytest.mark.parametrize("seed", range(8))
def test_contraction_equals_round_fixed_point(seed):
    H, R, eta, _, _ = _random_level_inputs(seed, ties=seed % 3 == 0)
    Ru = D.update_resistance(H.eptr, H.pins, R, eta)
    order = D.sort_order(Ru)
    sizes = np.diff(H.eptr)
    delta = D.quantile_threshold(Ru, sizes, 0.6)
    owner, contracted = D.contract(H.n, H.eptr, H.pins, order, Ru, delta)
    rank = np.empty(H.m, dtype=np.int64)
    rank[order] = np.arange(H.m)
    cand = (sizes >= 2) & (Ru < delta)
    assert np.array_equal(contracted, _greedy_rounds(H.n, H.eptr, H.pins, rank, cand))
    # defining properties: pin-disjoint, maximal in the order, owners consistent
    for e in np.flatnonzero(cand):
        ps = H.pins[H.eptr[e]:H.eptr[e + 1]]
        if contracted[e]:
            assert (owner[ps] == e).all()
        else:
            blockers = owner[ps]
            assert (blockers >= 0).any() and (rank[blockers[blockers >= 0]] < rank[e]).any()
    assert not contracted[~cand].any()


@pytest.mark.parametrize("seed", range(4))
def test_clusters_and_weights(seed):
    H, R, eta, _, _ = _random_level_inputs(seed)
    Ru = D.update_resistance(H.eptr, H.pins, R, eta)
    order = D.sort_order(Ru)
    owner, contracted = D.contract(H.n, H.eptr, H.pins, order, Ru,
                                   D.quantile_threshold(Ru, np.diff(H.eptr), 0.5))
    cluster, nc, eta_next, formed_by = D.clusters(H.n, H.eptr, H.pins, owner, contracted, Ru, eta)
    assert sorted(set(cluster.tolist())) == list(range(nc))
    firsts = [int(np.flatnonzero(cluster == c)[0]) for c in range(nc)]
    assert firsts == sorted(firsts)  # numbered by smallest member
    for c in range(nc):
        members = set(np.flatnonzero(cluster == c).tolist())
        e = formed_by[c]
        if e >= 0:
            assert members == set(H.pins[H.eptr[e]:H.eptr[e + 1]].tolist())
            assert eta_next[c] == Ru[e]
        else:
            assert len(members) == 1 and eta_next[c] == eta[members.pop()]


@pytest.mark.parametrize("seed", range(4))
def test_local_clustering_matches_vectorised_search(seed):
    H, R, eta, Q, QH = _random_level_inputs(seed, K=6)
    QH[seed % 6] = 0.0  # a column that takes no part
    out = D.level(H.n, H.eptr, H.pins, H.w, R, Q, QH, eta, q=0.4)
    cluster, formed_by = out["cluster"], out["formed_by"]
    nc = len(formed_by)
    # centroids by numpy means, distances for every (vertex, cluster) pair at once
    mu = np.zeros((nc, Q.shape[1]))
    for c in range(nc):
        mu[c] = Q[cluster == c].mean(axis=0)
    use = QH > 1e-300
    d_all = (((Q[:, None, use] - mu[None, :, use]) ** 2) / QH[None, use]).max(axis=2)
    for p in range(H.n):
        if out["owner"][p] >= 0:
            assert out["target"][p] == -1
            continue
        es = [e for e in range(H.m) if p in H.pins[H.eptr[e]:H.eptr[e + 1]]]
        cands = {int(cluster[u]) for e in es for u in H.pins[H.eptr[e]:H.eptr[e + 1]]
                 if u != p and formed_by[cluster[u]] >= 0}
        if not cands:
            assert out["target"][p] == -1
            continue
        cl = sorted(cands)
        best = cl[int(np.argmin(d_all[p, cl]))]
        assert out["target"][p] == best
        assert math.isclose(out["dist"][p], d_all[p, best], rel_tol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_coarse_hypergraph_by_set_algebra(seed):
    H, R, eta, Q, QH = _random_level_inputs(seed)
    out = D.level(H.n, H.eptr, H.pins, H.w, R, Q, QH, eta, q=0.7)
    final = out["final"]
    kept = set(out["emap"].tolist())
    for e in range(H.m):
        cl = set(final[H.pins[H.eptr[e]:H.eptr[e + 1]]].tolist())
        assert (len(cl) >= 2) == (e in kept)
    assert out["emap"].tolist() == sorted(kept)
    for i, e in enumerate(out["emap"]):
        ps = out["pins"][out["eptr"][i]:out["eptr"][i + 1]].tolist()
        assert len(ps) == len(set(ps)) >= 2
        assert set(ps) == set(final[H.pins[H.eptr[e]:H.eptr[e + 1]]].tolist())
        assert out["w"][i] == H.w[e]
    # weights: every fine vertex's weight and every contraction's resistance
    # reach exactly one final cluster, plus the seeds' distances
    total = eta.sum() + out["R_upd"][out["contracted"]].sum() \
        - sum(eta[H.pins[H.eptr[e]:H.eptr[e + 1]]].sum() for e in np.flatnonzero(out["contracted"])) \
        + out["dist"][out["target"] >= 0].sum()
    assert math.isclose(out["eta"].sum(), total, rel_tol=1e-12)
