"""Pins of the oracle's two variants of Algorithm 1 (Section III-A.3):

* the Krylov pool of one expansion only (ops="star" is the earlier HyperEF
  method, which the paper contrasts with the mixed pool): its columns span
  the same nested spaces as the raw power basis M^j x of that expansion,
  checked through LAPACK QR, and they are the corresponding columns of the
  mixed pool;
* EMBED scoring (reading A7's alternative: p, q the pins farthest apart in
  the whole embedding): the pair agrees with scipy's pdist, and the scores
  obey what the definitions force: equal to the per-vector max-min scores on
  2-pin hyperedges and for a one-column basis, never above them otherwise."""
import numpy as np
import pytest
from scipy.spatial.distance import pdist

from netlists import start_block
from oracle import hef_oracle as O
from tests._hypergraphs import random_hypergraph


def small_case(seed, n=40, m=60, kmax=5, S=2):
    H = random_hypergraph(n, m, kmax, seed, weights=True)
    x0c, x0b = start_block(H.n, H.m, S, seed)
    return H, x0c, x0b


@pytest.mark.parametrize("ops,op", [("star", O.STAR), ("clique", O.CLIQUE)])
def test_single_expansion_pool_is_the_matching_columns(ops, op):
    H, x0c, x0b = small_case(1)
    k, S = 3, 2
    both = O.krylov_basis(H.n, H.eptr, H.pins, H.w, x0c, x0b, k)
    one = O.krylov_basis(H.n, H.eptr, H.pins, H.w, x0c, x0b, k, ops=ops)
    assert one.shape == (H.n, k * S)
    for j in range(k):
        for s in range(S):
            assert np.array_equal(one[:, j * S + s], both[:, j * 2 * S + op * S + s])


def test_star_pool_spans_raw_power_basis():
    H, x0c, x0b = small_case(2, n=30, m=45, S=1)
    k = 3
    V = O.krylov_basis(H.n, H.eptr, H.pins, H.w, x0c, x0b, k, ops="star")
    Mb, db = O.random_walk(O.star_expansion(H.n, H.eptr, H.pins, H.w))
    tb = O.trivial_vectors(O.STAR, H.n, db)
    x = O.deflate(x0b[:, 0].copy(), db, tb)
    P = []
    for _ in range(k):
        x = Mb @ x
        col = x[:H.n]
        P.append(col - col.mean())
    P = np.array(P).T
    for j in range(1, k + 1):  # nested spans: the first j columns of each
        qa, _ = np.linalg.qr(V[:, :j])
        qb, _ = np.linalg.qr(P[:, :j])
        sv = np.linalg.svd(qa.T @ qb, compute_uv=False)
        assert sv.min() > 1 - 1e-10, (j, sv)


@pytest.mark.parametrize("seed", range(5))
def test_embed_pair_agrees_with_pdist(seed):
    rng = np.random.default_rng(seed)
    H = random_hypergraph(50, 80, 9, seed)
    Q = rng.standard_normal((H.n, 7))
    p, q = O.embed_pairs(Q, H.eptr, H.pins)
    for e in range(H.m):
        pe = H.pins[H.eptr[e]:H.eptr[e + 1]]
        t = int(np.argmax(pdist(Q[pe])))
        ia, ib = np.triu_indices(len(pe), 1)
        assert (p[e], q[e]) == (pe[ia[t]], pe[ib[t]])


@pytest.mark.parametrize("seed", range(4))
def test_embed_scores_against_max_min_scores(seed):
    rng = np.random.default_rng(seed)
    H = random_hypergraph(60, 90, 6, seed, weights=True)
    Q = rng.standard_normal((H.n, 5))
    emb = O.edge_resistance_embed(Q, H.eptr, H.pins, H.w)
    ref = O.edge_resistance(Q, H.eptr, H.pins, H.w)
    assert np.array_equal(emb["QH"], ref["QH"])  # Eq. non-linerQ is unchanged
    sizes = np.diff(H.eptr)
    two = sizes == 2
    assert np.allclose(emb["R"][two], ref["R"][two], rtol=1e-15, atol=0)
    assert (emb["R"] <= ref["R"] * (1 + 1e-14)).all()
    # one column: the farthest pair is the arg-max / arg-min pair
    Q1 = Q[:, :1]
    e1 = O.edge_resistance_embed(Q1, H.eptr, H.pins, H.w)
    r1 = O.edge_resistance(Q1, H.eptr, H.pins, H.w)
    assert np.allclose(e1["R"], r1["R"], rtol=1e-15, atol=0)
