"""Plain FP64 CPU oracle of the hyperedge effective-resistance estimator of
HyperEF 2.0 (Algorithm 1, Section III-A.3).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg; the GPU path never imports it and the two share
no code.  Everything is numpy/scipy in float64, written to be checked by eye
against the paper rather than to be fast.

Method, in the paper's order (Algorithm 1):

1. Star expansion G_b (step 1): a bipartite graph on |V| + |E| vertices with an
   edge (p, e) of weight z_b(e, p) = w(e)/d(e) for every pin p of hyperedge e.
2. Clique expansion G_c (step 2): every pin pair of e joined with weight
   w(e)/(|e|-1) (default) or w(e)/C(|e|,2) (``clique="paper"``).
3. Krylov vectors (step 3, Eq. krylov): for each expansion and each random
   start x, the vectors A x, A^2 x, ..., A^k x with A the random-walk
   normalised adjacency D^-1 W; only node entries are kept (star-node entries
   removed) and each vector is taken modulo the all-ones vector.
4. Gram-Schmidt (step 4): orthonormal chi^(1..K) in canonical column order.
5. Ratios (step 5, Eqs. non-linerQ and ratios) and R_e = max over i (Eq. R).

Readings where the paper is silent (each listed in the design notes):
 * d(e) in z_b = w(e)/d(e) is the pin count |e|;
 * "normalised adjacency" is the random walk M = D^-1 W, whose trivial
   eigenvectors (the constant on non-isolated vertices for both expansions and,
   for the bipartite star expansion, the vertex/star-node constants) are
   deflated from the start vector in the degree-weighted inner product; M
   commutes with that projector, so every Krylov vector stays deflated;
 * the chain for order k keeps A x ... A^k x (the raw random x is not part of
   the basis);
 * p, q in Eq. ratios are the arg-max / arg-min pins of chi^(i) on e, so
   (chi^T b_pq)^2 is the squared spread of chi^(i) over e;
 * hyperedges with fewer than 2 pins join neither expansion and score 0;
   vertices of degree 0 have zero rows in M;
 * a basis column whose norm after orthogonalisation falls below 1e-12 of its
   norm before is rank-deficient and dropped; a column with Q_H <= 1e-300 is
   skipped in the max.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

CLIQUE = 0
STAR = 1

DROP_TOL = 1e-12
QH_TINY = 1e-300


# ----------------------------------------------------------------------------
# Section II / III-A.3: expansions and their random-walk operators


def edge_sizes(eptr):
    return np.diff(np.asarray(eptr, dtype=np.int64))


def clique_expansion(n, eptr, pins, w, clique="hyperedge"):
    """Adjacency W_c of the clique expansion G_c (Section III-A.3).

    Every unordered pin pair {u, v} of a hyperedge e with |e| >= 2 receives
    weight w(e)/(|e|-1) (``clique="hyperedge"``) or w(e)/C(|e|,2)
    (``clique="paper"``); contributions of different hyperedges add.
    """
    sizes = edge_sizes(eptr)
    rows, cols, vals = [], [], []
    for e in range(sizes.size):
        k = int(sizes[e])
        if k < 2:
            continue
        pe = pins[eptr[e]:eptr[e + 1]].astype(np.int64)
        if clique == "hyperedge":
            zc = w[e] / (k - 1)
        elif clique == "paper":
            zc = w[e] / (k * (k - 1) / 2.0)
        else:
            raise ValueError(clique)
        u = np.repeat(pe, k)
        v = np.tile(pe, k)
        off = u != v
        rows.append(u[off])
        cols.append(v[off])
        vals.append(np.full(int(off.sum()), zc))
    if rows:
        rows = np.concatenate(rows)
        cols = np.concatenate(cols)
        vals = np.concatenate(vals)
    else:
        rows = cols = np.zeros(0, np.int64)
        vals = np.zeros(0)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def star_expansion(n, eptr, pins, w):
    """Adjacency W_b of the star (bipartite) expansion G_b on n + m vertices
    (Section III-A.3): vertex p and star node n+e are joined with weight
    z_b(e, p) = w(e)/|e| for each pin p of hyperedge e with |e| >= 2."""
    sizes = edge_sizes(eptr)
    m = sizes.size
    rows, cols, vals = [], [], []
    for e in range(m):
        k = int(sizes[e])
        if k < 2:
            continue
        pe = pins[eptr[e]:eptr[e + 1]].astype(np.int64)
        z = w[e] / k
        rows += [pe, np.full(k, n + e)]
        cols += [np.full(k, n + e), pe]
        vals += [np.full(k, z), np.full(k, z)]
    if rows:
        rows = np.concatenate(rows)
        cols = np.concatenate(cols)
        vals = np.concatenate(vals)
    else:
        rows = cols = np.zeros(0, np.int64)
        vals = np.zeros(0)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n + m, n + m))


def laplacian(W):
    """L = D - A (Eq. di_adjacency and the line after it)."""
    d = np.asarray(W.sum(axis=1)).ravel()
    return sp.diags(d) - W


def random_walk(W):
    """Normalised adjacency M = D^-1 W; rows of degree-0 vertices are zero.
    Returns (M, d)."""
    d = np.asarray(W.sum(axis=1)).ravel()
    dinv = np.zeros_like(d)
    nz = d > 0
    dinv[nz] = 1.0 / d[nz]
    return sp.diags(dinv) @ W, d


def trivial_vectors(op, n, d):
    """Eigenvectors of M with |eigenvalue| = 1 that every random-walk Krylov
    space contains regardless of the graph: the constant on the non-isolated
    vertices (eigenvalue 1), and for the bipartite star expansion also the
    +1/-1 vector over vertex/star-node sides (eigenvalue -1).  Returned as the
    side indicators, which span the same space."""
    active = (d > 0).astype(np.float64)
    if op == CLIQUE:
        return [active]
    t_v = active.copy()
    t_v[n:] = 0.0
    t_e = active.copy()
    t_e[:n] = 0.0
    return [t for t in (t_v, t_e) if t.any()]


def deflate(x, d, trivial):
    """Projection off the trivial eigenvectors in the degree-weighted inner
    product <a, b>_D = sum d_v a_v b_v (the one in which M is self-adjoint)."""
    x = x.copy()
    for t in trivial:
        den = float(np.dot(t * d, t))
        if den > 0:
            x -= t * (float(np.dot(t * d, x)) / den)
    return x


# ----------------------------------------------------------------------------
# Algorithm 1 step 3 / Eq. krylov: one Krylov chain


def krylov_chain(M, d, trivial, x0, k):
    """Vectors spanning, one at a time, span(A x, ..., A^j x) for j = 1..k
    with A = M and x = the deflated start x0.

    Each new vector is M times the previous one, made orthogonal to the
    earlier vectors of the same chain by classical Gram-Schmidt applied twice,
    and normalised.  Subtracting earlier chain vectors does not change the
    nested spans, so the result is the Krylov sequence itself, only better
    conditioned.  A vector that vanishes under orthogonalisation (the Krylov
    space is exhausted) is returned as zero.
    Returns an array (N, k)."""
    N = x0.shape[0]
    X = np.zeros((N, k))
    prev = deflate(x0, d, trivial)
    for j in range(k):
        y = M @ prev
        y = deflate(y, d, trivial)
        B = X[:, :j]
        for _ in range(2):  # Gram-Schmidt twice against the chain so far
            y -= B @ (B.T @ y)
        after = np.linalg.norm(y)
        if after <= DROP_TOL * np.linalg.norm(prev):
            # exhausted: M maps the chain into its own span (up to rounding),
            # so no later power adds a direction
            break
        y /= after
        X[:, j] = y
        prev = y
    return X


def krylov_basis(H_n, eptr, pins, w, x0_c, x0_b, k, clique="hyperedge", ops="both"):
    """The n x K matrix V (K = 2 k S) of Algorithm 1 step 3.

    Column c = (j-1)*2S + op*S + s holds the vertex entries of the j-th chain
    vector of start s of expansion op (0 = clique, 1 = star), with its mean
    removed (vectors are taken modulo the all-ones vector: scores only see
    differences).  Star-node entries are dropped (Section III-A.3).

    ops="star" (or "clique") keeps the pool of one expansion only (K = k S,
    column (j-1)*S + s): the star-only pool is the earlier HyperEF method
    that Section III-A.3 contrasts with the mixed pool."""
    n = H_n
    S = x0_c.shape[1]
    chosen = {"both": (CLIQUE, STAR), "clique": (CLIQUE,), "star": (STAR,)}[ops]
    Mc, dc = random_walk(clique_expansion(n, eptr, pins, w, clique))
    Mb, db = random_walk(star_expansion(n, eptr, pins, w))
    tc = trivial_vectors(CLIQUE, n, dc)
    tb = trivial_vectors(STAR, n, db)
    nop = len(chosen)
    K = nop * k * S
    V = np.zeros((n, K))
    for s in range(S):
        chains = {}
        if CLIQUE in chosen:
            chains[CLIQUE] = krylov_chain(Mc, dc, tc, x0_c[:, s], k)
        if STAR in chosen:
            chains[STAR] = krylov_chain(Mb, db, tb, x0_b[:, s], k)
        for j in range(k):
            for slot, op in enumerate(chosen):
                col = chains[op][:n, j]
                V[:, j * nop * S + slot * S + s] = col - col.mean()
    return V


# ----------------------------------------------------------------------------
# Algorithm 1 step 4: Gram-Schmidt


def gram_schmidt(V):
    """Classical Gram-Schmidt applied twice ("twice is enough"), column by
    column in the given order, giving Q with orthonormal columns and
    upper-triangular R with a positive diagonal (V = Q R).  A column whose
    norm after orthogonalisation is <= 1e-12 of its norm before is
    rank-deficient: its Q column is zero and it is marked False in ``kept``.
    Returns (Q, R, kept)."""
    n, K = V.shape
    Q = np.zeros((n, K))
    R = np.zeros((K, K))
    kept = np.zeros(K, dtype=bool)
    for i in range(K):
        y = V[:, i].copy()
        before = np.linalg.norm(y)
        B = Q[:, :i]
        for _ in range(2):
            c = B.T @ y
            R[:i, i] += c
            y -= B @ c
        after = np.linalg.norm(y)
        if before > 0 and after > DROP_TOL * before:
            Q[:, i] = y / after
            R[i, i] = after
            kept[i] = True
        else:
            R[:i, i] = 0.0
    return Q, R, kept


# ----------------------------------------------------------------------------
# Algorithm 1 steps 5 and 7: Eqs. non-linerQ, ratios and R


def spreads(Q, eptr, pins, chunk=4096):
    """For every hyperedge e and column i: max_{p in e} Q[p,i] - min_{p in e}
    Q[p,i], with the arg-max and arg-min pins (lowest position in e on ties).
    Hyperedges with < 2 pins get spread 0 and pins -1.  Segmented max/min use
    numpy's reduceat over blocks of hyperedges.
    Returns (spread (m,K), pmax (m,K), pmin (m,K))."""
    eptr = np.asarray(eptr, dtype=np.int64)
    pins = np.asarray(pins, dtype=np.int64)
    m = eptr.size - 1
    K = Q.shape[1]
    sp_ = np.zeros((m, K))
    pmax = np.full((m, K), -1, dtype=np.int64)
    pmin = np.full((m, K), -1, dtype=np.int64)
    sizes = np.diff(eptr)
    for e0 in range(0, m, chunk):
        e1 = min(m, e0 + chunk)
        sel = np.arange(e0, e1)[sizes[e0:e1] >= 2]
        if sel.size == 0:
            continue
        lens = sizes[sel]
        # pins of the selected hyperedges only, so each segment is contiguous
        rows = np.concatenate([np.arange(eptr[e], eptr[e + 1]) for e in sel])
        X = Q[pins[rows], :]
        starts = np.zeros(sel.size, dtype=np.int64)
        starts[1:] = np.cumsum(lens)[:-1]
        mx = np.maximum.reduceat(X, starts, axis=0)
        mn = np.minimum.reduceat(X, starts, axis=0)
        # first position attaining the max / min inside each hyperedge
        seg = np.repeat(np.arange(sel.size), lens)
        pos = np.arange(rows.size)[:, None] * np.ones((1, K), np.int64)
        big = np.int64(1) << 62
        fmax = np.minimum.reduceat(np.where(X == mx[seg], pos, big), starts, axis=0)
        fmin = np.minimum.reduceat(np.where(X == mn[seg], pos, big), starts, axis=0)
        sp_[sel] = mx - mn
        pmax[sel] = pins[rows[fmax]]
        pmin[sel] = pins[rows[fmin]]
    return sp_, pmax, pmin


def spreads_loop(Q, eptr, pins):
    """Same as ``spreads``, one hyperedge at a time (for small cases)."""
    m = len(eptr) - 1
    K = Q.shape[1]
    sp_ = np.zeros((m, K))
    pmax = np.full((m, K), -1, dtype=np.int64)
    pmin = np.full((m, K), -1, dtype=np.int64)
    for e in range(m):
        a, b = int(eptr[e]), int(eptr[e + 1])
        if b - a < 2:
            continue
        pe = np.asarray(pins[a:b], dtype=np.int64)
        X = Q[pe, :]
        imax = np.argmax(X, axis=0)  # first occurrence on ties
        imin = np.argmin(X, axis=0)
        cols = np.arange(K)
        sp_[e] = X[imax, cols] - X[imin, cols]
        pmax[e] = pe[imax]
        pmin[e] = pe[imin]
    return sp_, pmax, pmin


def quadratic_form(spread, w):
    """Q_H(chi^(i)) = sum_e w_e max_{u,v in e} (chi_u - chi_v)^2
    (Eq. non-linerQ), for every column i."""
    return (w[:, None] * spread ** 2).sum(axis=0)


def edge_resistance(Q, eptr, pins, w, reduce="max", kept=None):
    """Resistance ratios r_e(chi^(i)) = spread^2 / Q_H(chi^(i)) (Eq. ratios)
    and R_e = max_i r_e(chi^(i)) (Eq. R).

    ``reduce="sum"`` returns sum_i r_e instead (a test mode: with Laplacian
    eigenvectors as the basis it is the graph effective resistance of
    Eq. eff_resist0).  Columns with Q_H <= 1e-300 (or not in ``kept``) take no
    part.  Returns dict with R (m), QH (K), argvec (m, lowest i on ties,
    -1 when no column takes part), pmax/pmin (m, pins of column argvec)."""
    w = np.asarray(w, dtype=np.float64)
    spread, pmx, pmn = spreads(Q, eptr, pins)
    QH = quadratic_form(spread, w)
    K = Q.shape[1]
    use = QH > QH_TINY
    if kept is not None:
        use &= kept
    r = np.zeros_like(spread)
    r[:, use] = spread[:, use] ** 2 / QH[use]
    m = spread.shape[0]
    if reduce == "sum":
        R = r.sum(axis=1)
    else:
        R = r.max(axis=1) if K else np.zeros(m)
    rr = np.where(use[None, :], r, -1.0)
    argvec = np.argmax(rr, axis=1) if K else np.zeros(m, np.int64)
    none = ~use.any() if K else True
    sizes = edge_sizes(eptr)
    argvec = np.where((sizes >= 2) & (not none), argvec, -1)
    pmax = np.where(argvec >= 0, pmx[np.arange(m), np.maximum(argvec, 0)], -1)
    pmin = np.where(argvec >= 0, pmn[np.arange(m), np.maximum(argvec, 0)], -1)
    return dict(R=R, QH=QH, r=r, argvec=argvec, pmax=pmax, pmin=pmin, use=use)


def embed_pairs(Q, eptr, pins):
    """Reading A7's alternative for "p and q are the most distant nodes in the
    embedding space" (Eq. ratios): per hyperedge, the pair of pins farthest
    apart in the K-dimensional embedding, by squared Euclidean distance
    summed over the columns in ascending order (FP64); ties go to the first
    pair in (position of p, position of q) order, p before q in pin order.
    Returns (p, q) per hyperedge (-1 for hyperedges with < 2 pins)."""
    m = len(eptr) - 1
    K = Q.shape[1]
    pp = np.full(m, -1, dtype=np.int64)
    qq = np.full(m, -1, dtype=np.int64)
    for e in range(m):
        a, b = int(eptr[e]), int(eptr[e + 1])
        k = b - a
        if k < 2:
            continue
        ia, ib = np.triu_indices(k, 1)   # pairs in (a, b) lexicographic order
        X = Q[np.asarray(pins[a:b], dtype=np.int64), :].astype(np.float64)
        d = np.zeros(ia.size)
        for i in range(K):               # ascending columns, one rounding per step
            diff = X[ia, i] - X[ib, i]
            d = d + diff * diff
        t = int(np.argmax(d))            # first maximum
        pp[e] = pins[a + ia[t]]
        qq[e] = pins[a + ib[t]]
    return pp, qq


def edge_resistance_embed(Q, eptr, pins, w, kept=None):
    """Eq. ratios with p, q the embedding-farthest pair of ``embed_pairs``:
    r_e(chi^(i)) = (chi_p^(i) - chi_q^(i))^2 / Q_H(chi^(i)) with Q_H of Eq.
    non-linerQ (unchanged), R_e = max_i (Eq. R), argvec the lowest maximising
    column, pmax / pmin the pair ordered by their values in that column (p
    first when equal)."""
    w = np.asarray(w, dtype=np.float64)
    spread, _, _ = spreads(Q, eptr, pins)
    QH = quadratic_form(spread, w)
    use = QH > QH_TINY
    if kept is not None:
        use &= kept
    pp, qq = embed_pairs(Q, eptr, pins)
    m = len(eptr) - 1
    R = np.zeros(m)
    argvec = np.full(m, -1, dtype=np.int64)
    pmax = np.full(m, -1, dtype=np.int64)
    pmin = np.full(m, -1, dtype=np.int64)
    for e in range(m):
        if pp[e] < 0 or not use.any():
            continue
        best, bi = -1.0, -1
        for i in np.flatnonzero(use):
            diff = float(Q[pp[e], i]) - float(Q[qq[e], i])
            r = (diff * diff) / QH[i]
            if r > best:
                best, bi = r, int(i)
        R[e], argvec[e] = best, bi
        hi = Q[pp[e], bi] >= Q[qq[e], bi]
        pmax[e], pmin[e] = (pp[e], qq[e]) if hi else (qq[e], pp[e])
    return dict(R=R, QH=QH, argvec=argvec, pmax=pmax, pmin=pmin, use=use, p=pp, q=qq)


# ----------------------------------------------------------------------------
# Algorithm 1 end to end


def hyperedge_resistance(n, eptr, pins, w, x0_c, x0_b, k, clique="hyperedge",
                         reduce="max", ops="both"):
    """Algorithm 1: expansions, Krylov basis, Gram-Schmidt, ratios, max.
    ``ops`` selects the Krylov pool (see krylov_basis); reduce="embed" scores
    with the embedding-farthest pair (edge_resistance_embed).
    Returns the dict of ``edge_resistance`` plus V, Q, Rfac, kept."""
    eptr = np.asarray(eptr, dtype=np.int64)
    pins = np.asarray(pins, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    V = krylov_basis(n, eptr, pins, w, x0_c, x0_b, k, clique, ops)
    Q, Rf, kept = gram_schmidt(V)
    if reduce == "embed":
        out = edge_resistance_embed(Q, eptr, pins, w, kept)
    else:
        out = edge_resistance(Q, eptr, pins, w, reduce, kept)
    out.update(V=V, Q=Q, Rfac=Rf, kept=kept)
    return out
