"""Consumers of the hyperedge resistances: one coarsening level of HyperEF 2.0.

TEST INFRASTRUCTURE.  This module is the plain CPU statement that the GPU
kernels of the downstream calls are checked against, bit for bit.  Only
tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use it;
the library never does.  It shares no code with the library.

What it computes, in the order of Algorithm 2 (Section III-B, "Resistance-
Based Hypergraph Local Clustering") after Algorithm 1 (Section III-A.3):

  update_resistance   Eq. R_W_update: R_e <- sum_{v in e} eta(v) + R_e, where
                      eta(v) is the weight of the supernode v (zero on the
                      original hypergraph; Section III-A.3, "Multilevel
                      Effective Resistance Clustering").
  sort_order          Algorithm 1 step 6: hyperedges sorted by resistance.
  quantile_threshold  the contraction threshold delta (the paper gives none).
  contract            Algorithm 2 step 5: starting from the lowest resistance,
                      contract a hyperedge if R_e < delta.
  clusters            the supernodes formed by the contraction and their
                      weights (Section III-A.3: a supernode's weight is the
                      resistance of the hyperedge that formed it).
  local_clustering    Algorithm 2 steps 7-10 (Section III-B.2): isolated
                      vertices join the neighbouring supernode at the smallest
                      resistance distance, the supernode being represented by
                      the mean of its members' embedding vectors.
  coarsen             Algorithm 2 step 6: the coarse hypergraph H'.
  level               all of the above for one level.

Readings of the paper (it fixes none of these details):
  D1  Eq. R_W_update's sum runs over the hyperedge's pins in their given
      order, left to right from 0.0; R_e is added last.  All in FP64.
  D2  Ties in the sort are broken by ascending hyperedge id.
  D3  delta: given by the caller, or the q-quantile of the updated
      resistances of the hyperedges with at least 2 pins: the value at
      position floor(q (c - 1)) of their ascending order (c of them).  A
      hyperedge is contracted only if its updated resistance is < delta.
  D4  Contraction is greedy in sorted order: a hyperedge with at least two
      pins and R_e < delta is contracted if none of its pins already belongs
      to a hyperedge contracted before it; all its pins then form one
      supernode.  Each supernode is formed by exactly one hyperedge, so its
      weight (the resistance of that hyperedge) is well defined.  Vertices
      left out are the isolated (unclustered) vertices of Section III-B.2.
  D5  Cluster ids are assigned in ascending vertex order: a new id for each
      isolated vertex and for the smallest-id pin of each contracted
      hyperedge; the other pins take their supernode's id.  The weight of a
      supernode is the updated resistance of its hyperedge; an isolated
      vertex keeps its own weight.
  D6  Seeds (Algorithm 2 step 7) are the isolated vertices.  A seed's
      candidates (Eq. neighbors) are the supernodes of its co-pins in the
      hyperedges that contain it; only supernodes formed by a contraction are
      candidates, so seeds never join each other.  A seed with no candidate
      stays isolated.  All seeds choose at once, from the contraction's
      supernodes.
  D7  The distance between seed p and supernode c (Section III-B.2, "we reuse
      the vector chi ... to evaluate the numerator of Eq. ratios"): with the
      centroid mu_c[i] = (sum of Q[u, i] over the members u, in the forming
      hyperedge's pin order) / |c|, d(p, c) = max over columns i with
      Q_H[i] > 1e-300 of (Q[p, i] - mu_c[i])^2 / Q_H[i], the Eq. ratios term
      maximised over the basis as in Eq. R (0 when no column qualifies).  The
      seed joins the candidate with the smallest d, ties to the smallest
      cluster id.  FP64 throughout; Q is widened exactly from its storage
      type.
  D8  Step 10's update of the merged cluster's resistance data: the
      supernode's weight grows by eta(p) + d(p, c) for each seed p that joins
      it, added in ascending p order after its own weight.
  D9  After the merges, cluster ids are made compact again, numbered in the
      order of each final cluster's smallest vertex; the coarse hypergraph
      maps every pin to its cluster, keeps the first occurrence of each
      cluster in pin order, drops hyperedges left with fewer than 2 pins and
      keeps the others' weights and relative order.
"""
from __future__ import annotations

import math

import numpy as np


def update_resistance(eptr, pins, R, eta):
    """Eq. R_W_update (reading D1)."""
    m = len(eptr) - 1
    out = np.empty(m, dtype=np.float64)
    for e in range(m):
        acc = 0.0
        for t in range(int(eptr[e]), int(eptr[e + 1])):
            acc += float(eta[pins[t]])
        out[e] = acc + float(R[e])
    return out


def sort_order(Ru):
    """Algorithm 1 step 6 with reading D2: ids in ascending (Ru, id) order."""
    return np.array(sorted(range(len(Ru)), key=lambda e: (Ru[e], e)), dtype=np.int32)


def quantile_threshold(Ru, sizes, q):
    """Reading D3: the q-quantile of the updated resistances of hyperedges
    with at least 2 pins (+inf when there is none)."""
    vals = sorted(float(Ru[e]) for e in range(len(Ru)) if sizes[e] >= 2)
    if not vals:
        return math.inf
    return vals[int(math.floor(q * (len(vals) - 1)))]


def contract(n, eptr, pins, order, Ru, delta):
    """Algorithm 2 step 5 with reading D4.  Returns owner[n] (the contracted
    hyperedge that each vertex joined, or -1) and contracted[m] (bool)."""
    m = len(eptr) - 1
    owner = np.full(n, -1, dtype=np.int32)
    contracted = np.zeros(m, dtype=bool)
    for e in order:
        a, b = int(eptr[e]), int(eptr[e + 1])
        if b - a < 2 or not (Ru[e] < delta):
            continue
        ps = pins[a:b]
        if any(owner[p] >= 0 for p in ps):
            continue
        for p in ps:
            owner[p] = e
        contracted[e] = True
    return owner, contracted


def clusters(n, eptr, pins, owner, contracted, Ru, eta):
    """Reading D5.  Returns cluster[n], the number of clusters, the cluster
    weights eta_next[nc] and formed_by[nc] (forming hyperedge or -1)."""
    minpin = {}
    for e in np.flatnonzero(contracted):
        minpin[int(e)] = int(min(pins[int(eptr[e]):int(eptr[e + 1])]))
    cluster = np.full(n, -1, dtype=np.int32)
    nc = 0
    for v in range(n):
        if owner[v] < 0 or minpin[int(owner[v])] == v:
            cluster[v] = nc
            nc += 1
    eta_next = np.zeros(nc, dtype=np.float64)
    formed_by = np.full(nc, -1, dtype=np.int32)
    for v in range(n):
        if owner[v] >= 0:
            rep = minpin[int(owner[v])]
            cluster[v] = cluster[rep]
            if rep == v:
                eta_next[cluster[v]] = Ru[owner[v]]
                formed_by[cluster[v]] = owner[v]
        else:
            eta_next[cluster[v]] = eta[v]
    return cluster, nc, eta_next, formed_by


def centroid(c, eptr, pins, formed_by, Q):
    """Reading D7: mean embedding row of the contracted supernode c."""
    K = Q.shape[1]
    e = formed_by[c]
    a, b = int(eptr[e]), int(eptr[e + 1])
    mu = np.zeros(K, dtype=np.float64)
    for i in range(K):
        acc = 0.0
        for t in range(a, b):
            acc += float(Q[pins[t], i])
        mu[i] = acc / (b - a)
    return mu


def seed_distance(qp, mu_c, QH):
    """Reading D7: max over the usable columns of (q_p - mu_c)^2 / Q_H."""
    d = 0.0
    for i in range(len(QH)):
        if QH[i] > 1e-300:
            diff = float(qp[i]) - float(mu_c[i])
            r = (diff * diff) / float(QH[i])
            if r > d:
                d = r
    return d


def seed_choice(p, eptr, pins, vptr, vedge, cluster, formed_by, Q, QH, mu_cache=None):
    """Readings D6-D7 for one isolated vertex p: (supernode, distance), or
    (-1, 0.0) without a candidate.  mu_cache (dict) keeps centroids."""
    mu_cache = {} if mu_cache is None else mu_cache
    best, bd = -1, math.inf
    for t in range(int(vptr[p]), int(vptr[p + 1])):
        e = int(vedge[t])
        for s in range(int(eptr[e]), int(eptr[e + 1])):
            u = int(pins[s])
            c = int(cluster[u])
            if u == p or formed_by[c] < 0:
                continue
            if c not in mu_cache:
                mu_cache[c] = centroid(c, eptr, pins, formed_by, Q)
            d = seed_distance(Q[p], mu_cache[c], QH)
            if d < bd or (d == bd and c < best):
                best, bd = c, d
    return (best, bd) if best >= 0 else (-1, 0.0)


def local_clustering(n, eptr, pins, vptr, vedge, cluster, owner, formed_by, eta, eta_next, Q, QH):
    """Algorithm 2 steps 7-10 with readings D6-D8.  vptr/vedge: the hyperedges
    containing each vertex.  Returns target[n] (the supernode each seed joins,
    -1 otherwise), dist[n] and the updated supernode weights."""
    target = np.full(n, -1, dtype=np.int32)
    dist = np.zeros(n, dtype=np.float64)
    mu_cache = {}
    for p in range(n):
        if owner[p] >= 0:
            continue
        target[p], dist[p] = seed_choice(p, eptr, pins, vptr, vedge, cluster, formed_by, Q, QH,
                                         mu_cache)
    eta2 = eta_next.copy()
    for p in range(n):
        if target[p] >= 0:
            eta2[target[p]] += float(eta[p]) + float(dist[p])
    return target, dist, eta2


def final_clusters(n, cluster, target, eta2):
    """Reading D9: compact cluster ids after the merges and their weights."""
    rep_of = {}
    for v in range(n):
        c = int(target[v]) if target[v] >= 0 else int(cluster[v])
        rep_of.setdefault(c, v)
    out = np.full(n, -1, dtype=np.int32)
    newid = {}
    for v in range(n):
        c = int(target[v]) if target[v] >= 0 else int(cluster[v])
        if rep_of[c] == v:
            newid[c] = len(newid)
    for v in range(n):
        c = int(target[v]) if target[v] >= 0 else int(cluster[v])
        out[v] = newid[c]
    eta_f = np.zeros(len(newid), dtype=np.float64)
    for c, i in newid.items():
        eta_f[i] = eta2[c]
    return out, len(newid), eta_f


def coarsen(eptr, pins, w, cluster):
    """Algorithm 2 step 6 with reading D9: (eptr', pins', w', emap) where
    emap[e'] is the fine hyperedge that coarse hyperedge e' comes from."""
    m = len(eptr) - 1
    ce, cp, cw, emap = [0], [], [], []
    for e in range(m):
        seen = []
        for t in range(int(eptr[e]), int(eptr[e + 1])):
            c = int(cluster[pins[t]])
            if c not in seen:
                seen.append(c)
        if len(seen) >= 2:
            cp.extend(seen)
            ce.append(len(cp))
            cw.append(float(w[e]))
            emap.append(e)
    return (np.array(ce, dtype=np.int64), np.array(cp, dtype=np.int32),
            np.array(cw, dtype=np.float64), np.array(emap, dtype=np.int32))


def vertex_incidence(n, eptr, pins):
    """vptr[n+1], vedge[P]: the hyperedges containing each vertex, ascending."""
    m = len(eptr) - 1
    lists = [[] for _ in range(n)]
    for e in range(m):
        for t in range(int(eptr[e]), int(eptr[e + 1])):
            lists[int(pins[t])].append(e)
    vptr = np.zeros(n + 1, dtype=np.int64)
    vptr[1:] = np.cumsum([len(x) for x in lists])
    vedge = np.array([e for x in lists for e in x], dtype=np.int32)
    return vptr, vedge


def level(n, eptr, pins, w, R, Q, QH, eta=None, delta=None, q=0.5):
    """One level of Algorithm 2 (steps 4-10) from the scores of Algorithm 1."""
    m = len(eptr) - 1
    eta = np.zeros(n) if eta is None else np.asarray(eta, dtype=np.float64)
    sizes = np.diff(eptr)
    Ru = update_resistance(eptr, pins, R, eta)
    order = sort_order(Ru)
    if delta is None:
        delta = quantile_threshold(Ru, sizes, q)
    owner, contracted = contract(n, eptr, pins, order, Ru, delta)
    cluster, nc, eta_next, formed_by = clusters(n, eptr, pins, owner, contracted, Ru, eta)
    vptr, vedge = vertex_incidence(n, eptr, pins)
    target, dist, eta2 = local_clustering(n, eptr, pins, vptr, vedge, cluster, owner, formed_by,
                                          eta, eta_next, Q, QH)
    final, nf, eta_f = final_clusters(n, cluster, target, eta2)
    ce, cp, cw, emap = coarsen(eptr, pins, w, final)
    return dict(R_upd=Ru, order=order, delta=delta, owner=owner, contracted=contracted,
                cluster=cluster, nc=nc, eta_next=eta_next, formed_by=formed_by, target=target,
                dist=dist, final=final, nf=nf, eta=eta_f, eptr=ce, pins=cp, w=cw, emap=emap,
                m=m)
