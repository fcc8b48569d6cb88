"""Pins of the FP64 oracle against facts that do not come from the oracle
itself: closed forms, textbook constructions, invariants of the definitions
and brute force on tiny inputs.  CPU only."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from netlists import start_block, workload
from oracle import hef_oracle as O
from tests._hypergraphs import from_lists, random_graph, random_hypergraph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def _signed_incidence_laplacian(N, pairs, z):
    """Textbook L = B diag(z) B^T from an edge list (B = signed incidence)."""
    B = np.zeros((N, len(pairs)))
    for c, (u, v) in enumerate(pairs):
        B[u, c] = 1.0
        B[v, c] = -1.0
    return B @ np.diag(z) @ B.T


def _pairs_of(H, weight):
    pairs, z = [], []
    for e in range(H.m):
        pe = [int(p) for p in H.pins[H.eptr[e]:H.eptr[e + 1]]]
        k = len(pe)
        for a in range(k):
            for b in range(a + 1, k):
                pairs.append((pe[a], pe[b]))
                z.append(weight(H.w[e], k))
    return pairs, np.array(z)


# ---------------------------------------------------------------- expansions

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_laplacians_are_laplacians(seed):
    """Eq. di_adjacency: L = D - A has zero row sums and x^T L x >= 0."""
    H = random_hypergraph(30, 25, 6, seed, weights=True)
    rng = np.random.default_rng(seed)
    for W in (O.clique_expansion(H.n, H.eptr, H.pins, H.w),
              O.clique_expansion(H.n, H.eptr, H.pins, H.w, clique="paper"),
              O.star_expansion(H.n, H.eptr, H.pins, H.w)):
        L = O.laplacian(W).toarray()
        assert np.allclose(L, L.T)
        assert np.abs(L.sum(axis=1)).max() < 1e-13
        for _ in range(5):
            x = rng.standard_normal(L.shape[0])
            assert x @ L @ x >= -1e-12
        assert np.linalg.eigvalsh(L).min() > -1e-12


def test_clique_and_star_match_signed_incidence():
    """The expansions built from the adjacency equal the textbook Laplacian
    B Z B^T of their explicit pin-pair / pin-star edge lists."""
    H = random_hypergraph(25, 20, 7, 3, weights=True)
    for mode, wt in (("hyperedge", lambda w, k: w / (k - 1)),
                     ("paper", lambda w, k: w / (k * (k - 1) / 2))):
        pairs, z = _pairs_of(H, wt)
        Lref = _signed_incidence_laplacian(H.n, pairs, z)
        L = O.laplacian(O.clique_expansion(H.n, H.eptr, H.pins, H.w, mode)).toarray()
        assert np.allclose(L, Lref, atol=1e-13)
    pairs, z = [], []
    for e in range(H.m):
        pe = H.pins[H.eptr[e]:H.eptr[e + 1]]
        for p in pe:
            pairs.append((int(p), H.n + e))
            z.append(H.w[e] / len(pe))
    Lref = _signed_incidence_laplacian(H.n + H.m, pairs, np.array(z))
    L = O.laplacian(O.star_expansion(H.n, H.eptr, H.pins, H.w)).toarray()
    assert np.allclose(L, Lref, atol=1e-13)


def test_expansion_degrees_match_hypergraph_degree():
    """Section II defines d_v = sum_{e ∋ v} w(e).  With weight w/(|e|-1) each
    pin has |e|-1 clique neighbours, so the clique degree is d_v; the
    C(|e|,2) weighting spreads w(e) evenly over the pairs (Section III-A.3),
    so the clique weights of e sum to w(e); the star node of e has degree
    |e| * w(e)/|e| = w(e)."""
    H = random_hypergraph(40, 30, 9, 5, weights=True)
    dv = np.zeros(H.n)
    for e in range(H.m):
        dv[H.pins[H.eptr[e]:H.eptr[e + 1]]] += H.w[e]
    Wc = O.clique_expansion(H.n, H.eptr, H.pins, H.w)
    assert np.allclose(np.asarray(Wc.sum(axis=1)).ravel(), dv)
    Wp = O.clique_expansion(H.n, H.eptr, H.pins, H.w, clique="paper")
    assert np.isclose(Wp.sum() / 2, H.w.sum())
    Wb = O.star_expansion(H.n, H.eptr, H.pins, H.w)
    assert np.allclose(np.asarray(Wb.sum(axis=1)).ravel()[H.n:], H.w)


def test_two_pin_graph_both_clique_weights_coincide():
    """For |e| = 2, w/(|e|-1) = w/C(|e|,2) = w: the clique expansion is the
    graph itself."""
    G = random_graph(20, 40, 7)
    a = O.clique_expansion(G.n, G.eptr, G.pins, G.w).toarray()
    b = O.clique_expansion(G.n, G.eptr, G.pins, G.w, clique="paper").toarray()
    pairs, z = _pairs_of(G, lambda w, k: w)
    assert np.allclose(a, b)
    assert np.allclose(np.diag(a.sum(1)) - a, _signed_incidence_laplacian(G.n, pairs, z))


def test_random_walk_properties_and_deflation_commutes():
    """M = D^-1 W: M 1 = 1 on non-isolated rows, D M is symmetric, the
    trivial vectors are eigenvectors with eigenvalue +1 (and -1 for the
    bipartite star side vector), and the D-orthogonal deflation commutes
    with M."""
    H = random_hypergraph(30, 22, 6, 11, weights=True)
    # add an isolated vertex and a 1-pin hyperedge
    H = from_lists(H.n + 1, [list(H.pins[H.eptr[e]:H.eptr[e + 1]]) for e in range(H.m)] + [[3]],
                   list(H.w) + [1.5])
    rng = np.random.default_rng(0)
    for op, W in ((O.CLIQUE, O.clique_expansion(H.n, H.eptr, H.pins, H.w)),
                  (O.STAR, O.star_expansion(H.n, H.eptr, H.pins, H.w))):
        M, d = O.random_walk(W)
        Md = M.toarray()
        act = d > 0
        assert not act.all()  # isolated vertex / star node present
        assert np.allclose(Md.sum(1)[act], 1.0)
        assert np.allclose(Md.sum(1)[~act], 0.0)
        assert np.allclose(np.diag(d) @ Md, (np.diag(d) @ Md).T)
        triv = O.trivial_vectors(op, H.n, d)
        if op == O.CLIQUE:
            assert np.allclose(Md @ triv[0], triv[0])
        else:
            tv, te = triv
            assert np.allclose(Md @ (tv + te), tv + te)
            assert np.allclose(Md @ (tv - te), -(tv - te))
        for _ in range(3):
            x = rng.standard_normal(Md.shape[0])
            assert np.allclose(O.deflate(Md @ x, d, triv), Md @ O.deflate(x, d, triv))
            y = O.deflate(x, d, triv)
            assert np.allclose(O.deflate(y, d, triv), y)


# ---------------------------------------------------------------- Krylov

def test_single_hyperedge_closed_form():
    """One hyperedge on all n vertices: the clique walk is (J - I)/(n-1), so
    M x = -x/(n-1) for x ⊥ 1 and each clique chain spans one direction; the
    deflated star start is annihilated by the star walk.  Every basis vector
    then has Q_H = w spread^2, hence R = 1/w (golden file)."""
    g = json.load(open(GOLDEN))["single_hyperedge"]
    H = from_lists(g["n"], g["edges"], g["w"])
    Mc, dc = O.random_walk(O.clique_expansion(H.n, H.eptr, H.pins, H.w))
    x = np.random.default_rng(0).standard_normal(H.n)
    x -= x.mean()
    assert np.allclose(Mc @ x, -x / (H.n - 1))
    x0c, x0b = start_block(H.n, H.m, 2, 0)
    out = O.hyperedge_resistance(H.n, H.eptr, H.pins, H.w, x0c, x0b, 3)
    assert out["kept"].sum() == 2  # one clique direction per start
    assert np.allclose(out["R"], g["R"], rtol=1e-12)


def _power_basis(H, x0c, x0b, k):
    """V from raw powers M^j x (no orthogonalisation), canonical order."""
    n = H.n
    S = x0c.shape[1]
    ops = []
    for op, W in ((O.CLIQUE, O.clique_expansion(n, H.eptr, H.pins, H.w)),
                  (O.STAR, O.star_expansion(n, H.eptr, H.pins, H.w))):
        M, d = O.random_walk(W)
        ops.append((M, d, O.trivial_vectors(op, n, d)))
    V = np.zeros((n, 2 * k * S))
    for s in range(S):
        for op, x0 in ((O.CLIQUE, x0c[:, s]), (O.STAR, x0b[:, s])):
            M, d, t = ops[op]
            y = O.deflate(x0, d, t)
            for j in range(k):
                y = M @ y
                col = y[:n]
                V[:, j * 2 * S + op * S + s] = col - col.mean()
    return V


def test_nested_span_invariance_power_basis():
    """Q depends only on the nested spans of the canonical column order: the
    raw power basis M x, M^2 x, M^3 x (no stabilisation) gives the same Q
    (up to column signs) as the oracle's stabilised chains.  Reference QR is
    LAPACK's."""
    H = random_hypergraph(40, 45, 5, 21, weights=True)
    x0c, x0b = start_block(H.n, H.m, 2, 9)
    k = 3
    out = O.hyperedge_resistance(H.n, H.eptr, H.pins, H.w, x0c, x0b, k)
    Vp = _power_basis(H, x0c, x0b, k)
    Qp, Rp = np.linalg.qr(Vp)
    Qp *= np.sign(np.diag(Rp))
    assert out["kept"].all()
    assert np.allclose(np.abs(np.sum(Qp * out["Q"], axis=0)), 1.0, atol=1e-9)
    ref = O.edge_resistance(Qp, H.eptr, H.pins, H.w)
    assert np.allclose(out["R"], ref["R"], rtol=1e-8, atol=0)


def test_krylov_columns_are_smoothed_vertex_vectors():
    """Columns of V are mean-free and (for the clique chain) vectors of the
    D-deflated Krylov space: each lies in span of raw powers up to its step."""
    H, k, S = workload("grid64x32_m2300")
    x0c, x0b = start_block(H.n, H.m, S, 0)
    V = O.krylov_basis(H.n, H.eptr, H.pins, H.w, x0c, x0b, 4)
    assert np.abs(V.sum(axis=0)).max() < 1e-10
    Vp = _power_basis(H, x0c, x0b, 4)
    for c in range(V.shape[1]):
        B = Vp[:, :c + 1]
        coef, *_ = np.linalg.lstsq(B, V[:, c], rcond=None)
        assert np.linalg.norm(B @ coef - V[:, c]) < 1e-8 * np.linalg.norm(V[:, c])


# ---------------------------------------------------------------- QR

def test_gram_schmidt_matches_lapack_qr():
    rng = np.random.default_rng(4)
    V = rng.standard_normal((300, 24))
    Q, R, kept = O.gram_schmidt(V)
    Ql, Rl = np.linalg.qr(V)
    sgn = np.sign(np.diag(Rl))
    assert kept.all()
    assert np.allclose(Q, Ql * sgn, atol=1e-12)
    assert np.allclose(R, Rl * sgn[:, None], atol=1e-12)
    assert np.allclose(Q.T @ Q, np.eye(24), atol=1e-13)
    assert np.allclose(Q @ R, V, atol=1e-12)


def test_gram_schmidt_drops_dependent_columns():
    rng = np.random.default_rng(5)
    V = rng.standard_normal((100, 6))
    V[:, 3] = 2 * V[:, 0] - V[:, 1]
    V[:, 5] = 0.0
    Q, R, kept = O.gram_schmidt(V)
    assert list(kept) == [True, True, True, False, True, False]
    assert np.allclose(Q[:, ~kept], 0)
    Qk = Q[:, kept]
    assert np.allclose(Qk.T @ Qk, np.eye(4), atol=1e-13)


# ---------------------------------------------------------------- scoring

def test_spreads_brute_force_and_ties():
    """max - min over a hyperedge equals the brute-force max over pin pairs
    of |x_u - x_v| (Eq. non-linerQ); arg-max/arg-min take the lowest
    position on ties."""
    H = random_hypergraph(20, 30, 6, 8)
    rng = np.random.default_rng(1)
    Q = np.round(rng.standard_normal((H.n, 7)), 1)  # rounding creates ties
    spv, pmx, pmn = O.spreads(Q, H.eptr, H.pins)
    spl, lmx, lmn = O.spreads_loop(Q, H.eptr, H.pins)
    assert np.array_equal(spv, spl) and np.array_equal(pmx, lmx) and np.array_equal(pmn, lmn)
    for e in range(H.m):
        pe = list(H.pins[H.eptr[e]:H.eptr[e + 1]])
        for i in range(Q.shape[1]):
            best = max(abs(Q[u, i] - Q[v, i]) for u in pe for v in pe)
            assert spv[e, i] == best
            col = [Q[p, i] for p in pe]
            first_max = pe[col.index(max(col))]
            first_min = pe[col.index(min(col))]
            assert pmx[e, i] == first_max and pmn[e, i] == first_min


@pytest.mark.parametrize("name_or_seed", ["grid64x32_m2300", 3, 4])
def test_weighted_ratio_sum_is_one(name_or_seed):
    """By Eq. non-linerQ, sum_e w_e r_e(chi) = sum_e w_e spread^2 / Q_H = 1 for
    every basis vector (Eq. ratios), hence 1 <= sum_e w_e R_e <= rank."""
    if isinstance(name_or_seed, str):
        H, k, S = workload(name_or_seed)
    else:
        H, k, S = random_hypergraph(60, 70, 8, name_or_seed, weights=True), 4, 2
    x0c, x0b = start_block(H.n, H.m, S, 1)
    out = O.hyperedge_resistance(H.n, H.eptr, H.pins, H.w, x0c, x0b, k)
    use = out["use"]
    sums = (H.w[:, None] * out["r"]).sum(axis=0)
    assert np.allclose(sums[use], 1.0, rtol=1e-12)
    tot = float((H.w * out["R"]).sum())
    assert 1.0 - 1e-12 <= tot <= use.sum() + 1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_two_pin_eigenbasis_gives_pinv_resistance_and_foster(seed):
    """Eq. eff_resist0: for a 2-pin graph and the Laplacian eigenbasis
    u_2..u_n, spread^2 = (u^T b_pq)^2 and Q_H(u_i) = u_i^T L u_i = lambda_i, so
    the summed ratios equal b^T L^+ b (pseudo-inverse) and
    sum_e w_e R_e = n - 1 (Foster).  The per-vector max is <= R_eff."""
    G = random_graph(25, 50, seed)
    pairs, z = _pairs_of(G, lambda w, k: w)
    L = _signed_incidence_laplacian(G.n, pairs, z)
    lam, U = np.linalg.eigh(L)
    U = U[:, 1:]
    Lp = np.linalg.pinv(L)
    reff = np.array([Lp[u, u] + Lp[v, v] - 2 * Lp[u, v] for u, v in pairs])
    s = O.edge_resistance(U, G.eptr, G.pins, G.w, reduce="sum")
    assert np.allclose(s["QH"], lam[1:], rtol=1e-10)
    assert np.allclose(s["R"], reff, rtol=1e-10)
    assert np.isclose((G.w * s["R"]).sum(), G.n - 1, rtol=1e-10)
    mx = O.edge_resistance(U, G.eptr, G.pins, G.w, reduce="max")
    assert (mx["R"] <= reff * (1 + 1e-12)).all()


@pytest.mark.parametrize("case", ["weighted_path", "triangle_plus_pendant"])
def test_golden_graphs_pinv_and_method_bound(case):
    """Hand-derived resistances (golden file) are reproduced through the
    eigenbasis route, and the Krylov estimate of Algorithm 1 never exceeds
    them (Eq. eff_resist0 is a max over all vectors)."""
    g = json.load(open(GOLDEN))[case]
    G = from_lists(g["n"], g["edges"], g["w"])
    pairs, z = _pairs_of(G, lambda w, k: w)
    L = _signed_incidence_laplacian(G.n, pairs, z)
    lam, U = np.linalg.eigh(L)
    s = O.edge_resistance(U[:, 1:], G.eptr, G.pins, G.w, reduce="sum")
    assert np.allclose(s["R"], g["R_eff"], rtol=1e-12)
    assert np.isclose((G.w * s["R"]).sum(), g["foster"])
    x0c, x0b = start_block(G.n, G.m, 1, 3)
    est = O.hyperedge_resistance(G.n, G.eptr, G.pins, G.w, x0c, x0b, 2)
    assert (est["R"] <= np.array(g["R_eff"]) * (1 + 1e-10)).all()


@pytest.mark.parametrize("seed", range(4))
def test_brute_force_bound_small_hypergraphs(seed):
    """On <= 12 vertices: with L2 the clique Laplacian of weights
    w/C(|e|,2), x^T L2 x <= Q_H(x) for all x (per hyperedge the pair sum is
    at most floor(k/2)ceil(k/2) spread^2), so every ratio is bounded by the
    generalised-eigenproblem maximum over span(Q) and by b^T L2^+ b, taken
    over all pin pairs of the hyperedge (enumerated)."""
    H = random_hypergraph(11, 9, 5, 100 + seed, weights=True)
    x0c, x0b = start_block(H.n, H.m, 2, seed)
    out = O.hyperedge_resistance(H.n, H.eptr, H.pins, H.w, x0c, x0b, 2)
    L2 = O.laplacian(O.clique_expansion(H.n, H.eptr, H.pins, H.w, "paper")).toarray()
    rng = np.random.default_rng(seed)
    for _ in range(20):
        x = rng.standard_normal(H.n)
        qh = sum(H.w[e] * max((x[u] - x[v]) ** 2 for u in H.pins[H.eptr[e]:H.eptr[e + 1]]
                              for v in H.pins[H.eptr[e]:H.eptr[e + 1]]) for e in range(H.m))
        assert x @ L2 @ x <= qh * (1 + 1e-12)
    Q = out["Q"][:, out["kept"]]
    A = Q.T @ L2 @ Q
    L2p = np.linalg.pinv(L2)
    for e in range(H.m):
        pe = list(H.pins[H.eptr[e]:H.eptr[e + 1]])
        span_max = full_max = 0.0
        for a in pe:
            for b in pe:
                if a == b:
                    continue
                bb = np.zeros(H.n)
                bb[a], bb[b] = 1.0, -1.0
                c = Q.T @ bb
                span_max = max(span_max, float(c @ np.linalg.solve(A, c)))
                full_max = max(full_max, float(bb @ L2p @ bb))
        assert out["R"][e] <= span_max * (1 + 1e-9) + 1e-15
        assert span_max <= full_max * (1 + 1e-9) + 1e-15


def test_degenerate_edges_and_isolated_vertices():
    """Hyperedges with < 2 pins score 0 and route nowhere; isolated vertices
    and a second component do not disturb the invariants."""
    H = from_lists(12, [[0, 1, 2], [2, 3], [4], [], [5, 6, 7], [6, 8], [1, 3]],
                   [1.0, 2.0, 1.0, 1.0, 0.5, 1.5, 1.0])
    x0c, x0b = start_block(H.n, H.m, 2, 4)
    out = O.hyperedge_resistance(H.n, H.eptr, H.pins, H.w, x0c, x0b, 3)
    a = O.spreads(out["Q"], H.eptr, H.pins)
    b = O.spreads_loop(out["Q"], H.eptr, H.pins)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert out["R"][2] == 0 and out["R"][3] == 0
    assert out["argvec"][2] == -1 and out["argvec"][3] == -1
    assert (out["R"] >= 0).all() and np.isfinite(out["R"]).all()
    sums = (H.w[:, None] * out["r"]).sum(axis=0)
    assert np.allclose(sums[out["use"]], 1.0)


def test_scores_invariant_to_sign_and_shift():
    H = random_hypergraph(30, 40, 6, 2, weights=True)
    rng = np.random.default_rng(6)
    Q = rng.standard_normal((H.n, 5))
    a = O.edge_resistance(Q, H.eptr, H.pins, H.w)
    Q2 = Q * np.array([1, -1, 1, -1, -1]) + rng.standard_normal(5)
    b = O.edge_resistance(Q2, H.eptr, H.pins, H.w)
    assert np.allclose(a["R"], b["R"], rtol=1e-12)
    assert np.array_equal(a["argvec"], b["argvec"])
