"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances: 1e-9 relative on every score >= 1e-3 of the largest in the FP64
form, 2e-3 in the FP32 form; Kendall tau >= 0.999 on the full ranking;
integer and index outputs (incidence order, routing) exact where they are
unique."""
import numpy as np
import pytest
import torch

from netlists import start_block, workload
from oracle import hef_oracle as O
from tests._gpu import DEV, kendall_tau, rel_errors, run_pipeline, to_dev
from tests._hypergraphs import from_lists, random_graph, random_hypergraph

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-9, torch.float32: 2e-3}


def hef():
    import paper_2511_06600_gb300 as m
    return m


# ---------------------------------------------------------------- incidence (a0)

@pytest.mark.parametrize("case", ["grid64x32_m2300", "degenerate", "random"])
def test_incidence_build_exact(case):
    if case == "grid64x32_m2300":
        H, _, _ = workload(case)
    elif case == "degenerate":
        H = from_lists(12, [[0, 1, 2], [2, 3], [4], [], [5, 6, 7], [6, 8], [1, 3], [11, 0]],
                       [1.0, 2.0, 1.0, 1.0, 0.5, 1.5, 1.0, 3.0])
    else:
        H = random_hypergraph(500, 700, 40, 7, weights=True, min_size=1)
    t = to_dev(H)
    inc = hef().build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    inc.check()
    ex = {k: v.cpu().numpy() for k, v in inc.export().items()}
    # locality order: ascending smallest pin, ties by caller id (stable)
    perm = ex["perm"]
    assert np.array_equal(np.sort(perm), np.arange(H.m))
    sizes = np.diff(H.eptr)
    key = np.array([H.pins[H.eptr[e]:H.eptr[e + 1]].min() if sizes[e] else 0 for e in range(H.m)])
    assert np.array_equal(perm, np.lexsort((np.arange(H.m), key)))
    # vertex-major incidence: each vertex's hyperedges, in locality order
    rank = np.empty(H.m, dtype=np.int64)
    rank[perm] = np.arange(H.m)
    edge_of = np.repeat(np.arange(H.m), sizes)
    for v in range(H.n):
        mine = edge_of[H.pins == v]
        expect = mine[np.argsort(rank[mine], kind="stable")]
        got = ex["vedge"][ex["vptr"][v]:ex["vptr"][v + 1]]
        assert np.array_equal(got, expect)
    # degrees of both expansions against the oracle's explicit adjacency
    Wc = O.clique_expansion(H.n, H.eptr, H.pins.astype(np.int64), H.w)
    Wb = O.star_expansion(H.n, H.eptr, H.pins.astype(np.int64), H.w)
    assert np.allclose(ex["dc"], np.asarray(Wc.sum(1)).ravel(), rtol=1e-14, atol=0)
    assert np.allclose(ex["db"], np.asarray(Wb.sum(1)).ravel()[:H.n], rtol=1e-14, atol=0)


@pytest.mark.parametrize("bad,bit", [("pin", 2), ("dup", 4), ("weight", 8), ("eptr", 1)])
def test_invalid_hypergraph_is_rejected(bad, bit):
    H = random_hypergraph(50, 40, 5, 3, weights=True)
    pins, w, eptr = H.pins.copy(), H.w.copy(), H.eptr.copy()
    if bad == "pin":
        pins[17] = H.n + 5
    elif bad == "dup":
        pins[H.eptr[9] + 1] = pins[H.eptr[9]]
    elif bad == "weight":
        w[5] = -1.0
    else:
        eptr[10] = eptr[11] + 1
    H2 = type(H)(n=H.n, eptr=eptr, pins=pins, w=w)
    x0c, x0b = start_block(H.n, H.m, 1, 0)
    t = to_dev(H2, x0c, x0b)
    h = hef()
    inc = h.build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    V = h.krylov_basis(inc, t["x0c"], t["x0b"], 2, torch.float64)  # must do no work, no fault
    out = h.edge_resistance(inc, V, 4)
    with pytest.raises(h.HefError) as ei:
        inc.check()
    assert ei.value.status == -7 and ei.value.detail & bit
    torch.cuda.synchronize()
    del out


@pytest.mark.parametrize("size,bad", [(20, None), (20, "dup"), (300, None), (300, "dup"),
                                      (300, "pin"), (700, None), (700, "dup")])
def test_long_hyperedge_validation(size, bad):
    """Pins of long hyperedges: duplicates found by the shared-memory hash
    (up to 512 pins) or the quadratic scan beyond, bad pins flagged, and a
    clean hypergraph accepted."""
    rng = np.random.default_rng(size)
    n = 1000
    sizes = [2, 3, size, 4, 2]
    edges = [rng.choice(n, k, replace=False).astype(np.int32) for k in sizes]
    if bad == "dup":
        edges[2][size - 1] = edges[2][size // 3]
    elif bad == "pin":
        edges[2][size // 2] = n + 7
    pins = np.concatenate(edges)
    eptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    w = np.ones(len(sizes))
    h = hef()
    t = {"eptr": torch.from_numpy(eptr).to(DEV), "pins": torch.from_numpy(pins).to(DEV),
         "w": torch.from_numpy(w).to(DEV)}
    inc = h.build_incidence(n, t["eptr"], t["pins"], t["w"])
    if bad is None:
        inc.check()
    else:
        with pytest.raises(h.HefError) as ei:
            inc.check()
        assert ei.value.status == -7 and ei.value.detail & (4 if bad == "dup" else 2)


def test_host_argument_errors():
    h = hef()
    H = random_hypergraph(30, 20, 4, 1)
    t = to_dev(H)
    with pytest.raises(h.HefError):
        h.build_incidence(0, t["eptr"], t["pins"], t["w"])
    inc = h.build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    x0c, x0b = start_block(H.n, H.m, 3, 0)
    td = to_dev(H, x0c, x0b)
    with pytest.raises(h.HefError):  # S = 3 unsupported
        h.krylov_basis(inc, td["x0c"], td["x0b"], 2, torch.float64)


# ---------------------------------------------------------------- Krylov (a1, a2)

@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("S,k", [(1, 10), (2, 3), (4, 5), (8, 2), (16, 1)])
def test_krylov_basis_spans_oracle_spaces(dtype, S, k):
    """Nested column spaces of V (mean removed) equal the oracle's: the QR of
    the GPU basis equals the oracle's Q up to column signs."""
    H = random_hypergraph(700, 650, 9, 11 + S, weights=True, min_size=1)
    x0c, x0b = start_block(H.n, H.m, S, S)
    t = to_dev(H, x0c, x0b)
    h = hef()
    inc = h.build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    V = h.krylov_basis(inc, t["x0c"], t["x0b"], k, dtype)
    inc.check()
    K = 2 * k * S
    Vg = V[:, :K].double().cpu().numpy()
    Vg = Vg - Vg.mean(axis=0)
    Qg, Rg = np.linalg.qr(Vg)
    ref = O.hyperedge_resistance(H.n, H.eptr, H.pins, H.w, x0c, x0b, k)
    assert ref["kept"].all()
    cos = np.abs(np.sum(Qg * ref["Q"], axis=0))
    tol = 1e-10 if dtype == torch.float64 else 1e-4
    assert np.abs(cos - 1).max() < tol


def test_krylov_exhausted_chain_gives_zero_columns():
    """Single hyperedge on all vertices: one clique direction per start, and
    the deflated star start is annihilated (zero columns)."""
    H = from_lists(7, [list(range(7))], [2.0])
    x0c, x0b = start_block(H.n, H.m, 2, 0)
    t = to_dev(H, x0c, x0b)
    h = hef()
    inc = h.build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    V = h.krylov_basis(inc, t["x0c"], t["x0b"], 3, torch.float64)[:, :12].cpu().numpy()
    norms = np.linalg.norm(V, axis=0)
    # columns: step j block = [clique s0, clique s1, star s0, star s1]
    assert (norms[:2] > 0.1).all()
    assert np.all(norms[2:] == 0)


# ---------------------------------------------------------------- CholQR2 (a3)

@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n,K", [(1000, 20), (4099, 160), (777, 33), (3000, 384), (257, 1)])
def test_orthonormalize_matches_lapack(dtype, n, K):
    rng = np.random.default_rng(n + K)
    V0 = rng.standard_normal((n, K)) + rng.standard_normal(K)  # nonzero means
    h = hef()
    ld = h.padded_ld(K, dtype)
    V = torch.zeros(n, ld, dtype=dtype, device=DEV)
    V[:, :K] = torch.from_numpy(V0).to(DEV, dtype)
    Q, R, rank = h.orthonormalize(V, K, want_R=True)
    torch.cuda.synchronize()
    Qn = Q[:, :K].double().cpu().numpy()
    assert int(rank.item()) == K
    Vc = V0.astype(np.float64) if dtype == torch.float64 else V0.astype(np.float32).astype(np.float64)
    Vc = Vc - Vc.mean(axis=0)
    Ql, Rl = np.linalg.qr(Vc)
    Ql *= np.sign(np.diag(Rl))
    tol = 1e-12 if dtype == torch.float64 else 2e-5
    assert np.abs(Qn - Ql).max() < tol * max(1.0, np.sqrt(K))
    assert np.abs(Qn.T @ Qn - np.eye(K)).max() < tol
    assert np.abs(Qn.sum(axis=0)).max() < tol * np.sqrt(n)
    Rg = R.cpu().numpy()
    assert np.allclose(Rg, Rl * np.sign(np.diag(Rl))[:, None], rtol=1e-6, atol=1e-6 * np.abs(Rl).max())


def test_orthonormalize_drops_dependent_columns():
    rng = np.random.default_rng(3)
    n, K = 500, 8
    V0 = rng.standard_normal((n, K))
    V0[:, 3] = 2 * V0[:, 0] - V0[:, 1] + 0.5     # dependent modulo constants
    V0[:, 6] = 7.0                              # constant: zero after mean removal
    h = hef()
    V = torch.from_numpy(V0).to(DEV).contiguous()
    Q, _, rank = h.orthonormalize(V, K)
    torch.cuda.synchronize()
    Qn = Q.cpu().numpy()
    ref_Q, _, kept = O.gram_schmidt(V0 - V0.mean(axis=0))
    assert int(rank.item()) == kept.sum() == 6
    assert np.all(Qn[:, ~kept] == 0)
    assert np.abs(np.abs(np.sum(Qn * ref_Q, axis=0))[kept] - 1).max() < 1e-12


# ---------------------------------------------------------------- scoring (a4, a5)

@pytest.mark.parametrize("K", [1, 20, 33, 160, 384])
def test_edge_resistance_on_oracle_basis(K):
    """The scorer alone, fed the same Q: scores to rounding, routing exact."""
    H = random_hypergraph(900, 1200, 30, K, weights=True, min_size=0)
    rng = np.random.default_rng(K)
    Q = rng.standard_normal((H.n, K))
    Q[:, 0] = 0.0  # an unused column (Q_H = 0)
    h = hef()
    t = to_dev(H)
    inc = h.build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    ld = h.padded_ld(K, torch.float64)
    Qd = torch.zeros(H.n, ld, dtype=torch.float64, device=DEV)
    Qd[:, :K] = torch.from_numpy(Q).to(DEV)
    out = h.edge_resistance(inc, Qd, K)
    inc.check()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    ref = O.edge_resistance(Q, H.eptr, H.pins, H.w)
    assert np.allclose(got["QH"], ref["QH"], rtol=1e-13, atol=0)
    assert np.allclose(got["R"], ref["R"], rtol=1e-12, atol=0)
    # routing is unique where the best ratio is clearly separated
    r = np.where(ref["use"][None, :], ref["r"], -1)
    srt = np.sort(r, axis=1)
    sep = (srt[:, -1] - srt[:, -2] > 1e-9 * np.abs(srt[:, -1])) if K > 1 else np.ones(H.m, bool)
    assert np.array_equal(got["argvec"][sep], ref["argvec"][sep])
    assert np.array_equal(got["pmax"][sep], ref["pmax"][sep])
    assert np.array_equal(got["pmin"][sep], ref["pmin"][sep])
    sizes = np.diff(H.eptr)
    assert np.all(got["R"][sizes < 2] == 0) and np.all(got["argvec"][sizes < 2] == -1)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("K,pad", [(20, 0), (20, 1), (33, 0), (160, 0)])
def test_edge_resistance_window_boundaries(dtype, K, pad):
    """Hyperedges of 0 to 200 pins (runs of empty ones; sizes around the 64
    pins a warp scores and the 96-slot windows the staged pass 1 copies),
    scored from shared-memory stages (16-byte row pitch) and by the gathering
    pass 1 (pad = 1: a pitch that is not a multiple of 16 bytes), against the
    oracle on the same Q."""
    rng = np.random.default_rng(100 * K + pad)
    n = 1500
    choices = np.array([0, 1, 2, 3, 5, 8, 40, 64, 65, 95, 96, 97, 200])
    prob = np.array([8, 4, 30, 20, 12, 8, 5, 3, 3, 2, 2, 2, 1], float)
    sizes = rng.choice(choices, size=700, p=prob / prob.sum())
    edges = [list(rng.choice(n, size=int(k), replace=False)) for k in sizes]
    H = from_lists(n, edges, rng.uniform(0.5, 2.0, size=len(edges)))
    Q = rng.standard_normal((n, K))
    if dtype == torch.float32:
        Q = Q.astype(np.float32).astype(np.float64)
    h = hef()
    t = to_dev(H)
    inc = h.build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    ld = h.padded_ld(K, dtype) + pad
    Qd = torch.zeros(n, ld, dtype=dtype, device=DEV)
    Qd[:, :K] = torch.from_numpy(Q).to(dtype).to(DEV)
    out = h.edge_resistance(inc, Qd, K)
    inc.check()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    ref = O.edge_resistance(Q, H.eptr, H.pins, H.w)
    # FP32: spreads are FP32 differences, Q_H partial sums FP32 per window
    rtol, sep_tol = (1e-12, 1e-9) if dtype == torch.float64 else (1e-5, 1e-4)
    assert np.allclose(got["QH"], ref["QH"], rtol=rtol, atol=0)
    assert np.allclose(got["R"], ref["R"], rtol=rtol, atol=0)
    r = np.where(ref["use"][None, :], ref["r"], -1)
    srt = np.sort(r, axis=1)
    sep = srt[:, -1] - srt[:, -2] > sep_tol * np.abs(srt[:, -1])
    assert sep.sum() > 0.9 * (sizes >= 2).sum()
    for key in ("argvec", "pmax", "pmin"):
        assert np.array_equal(got[key][sep], ref[key][sep]), key
    assert np.all(got["R"][sizes < 2] == 0) and np.all(got["argvec"][sizes < 2] == -1)


def test_edge_resistance_eigenbasis_closed_form():
    """Eq. eff_resist0 through the GPU scorer: 2-pin graph, Laplacian
    eigenvectors as the basis, summed ratios = pseudo-inverse resistance and
    Foster's sum n - 1."""
    G = random_graph(60, 150, 2)
    L = O.laplacian(O.clique_expansion(G.n, G.eptr, G.pins, G.w)).toarray()
    lam, U = np.linalg.eigh(L)
    U = np.ascontiguousarray(U[:, 1:])
    Lp = np.linalg.pinv(L)
    u, v = G.pins[0::2], G.pins[1::2]
    reff = Lp[u, u] + Lp[v, v] - 2 * Lp[u, v]
    h = hef()
    t = to_dev(G)
    inc = h.build_incidence(G.n, t["eptr"], t["pins"], t["w"])
    K = U.shape[1]
    ld = h.padded_ld(K, torch.float64)
    Qd = torch.zeros(G.n, ld, dtype=torch.float64, device=DEV)
    Qd[:, :K] = torch.from_numpy(U).to(DEV)
    out = h.edge_resistance(inc, Qd, K, reduce=h.HEF_REDUCE_SUM)
    R = out["R"].cpu().numpy()
    assert np.allclose(out["QH"].cpu().numpy(), lam[1:], rtol=1e-10)
    assert np.allclose(R, reff, rtol=1e-10)
    assert np.isclose((G.w * R).sum(), G.n - 1, rtol=1e-10)


# ---------------------------------------------------------------- end to end

@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_end_to_end_small_netlist(dtype):
    H, k, S = workload("grid64x32_m2300")
    x0c, x0b = start_block(H.n, H.m, S, 0)
    got = run_pipeline(H, x0c, x0b, k, dtype)
    ref = O.hyperedge_resistance(H.n, H.eptr, H.pins, H.w, x0c, x0b, k)
    err = rel_errors(got["R"], ref["R"])
    assert err["max"] <= TOL[dtype], err
    assert kendall_tau(got["R"], ref["R"]) >= 0.999
    assert np.allclose(got["QH"], ref["QH"], rtol=1e-8 if dtype == torch.float64 else 1e-4)
    # weighted ratio sum invariant on the GPU's own outputs
    assert 1.0 - 1e-6 <= float((H.w * got["R"]).sum()) <= got["rank"][0] + 1e-6


@pytest.mark.parametrize("clique_mode", [0, 1])
def test_end_to_end_degenerate_and_weighted(clique_mode):
    H = random_hypergraph(300, 420, 12, 5, weights=True, min_size=0)
    H = from_lists(H.n + 3, [list(H.pins[H.eptr[e]:H.eptr[e + 1]]) for e in range(H.m)],
                   H.w)  # three isolated vertices
    x0c, x0b = start_block(H.n, H.m, 2, 1)
    got = run_pipeline(H, x0c, x0b, 4, torch.float64, clique_mode=clique_mode)
    ref = O.hyperedge_resistance(H.n, H.eptr, H.pins, H.w, x0c, x0b, 4,
                                 clique="paper" if clique_mode else "hyperedge")
    assert rel_errors(got["R"], ref["R"])["max"] <= 1e-9
    sizes = np.diff(H.eptr)
    assert np.all(got["R"][sizes < 2] == 0)


def test_single_hyperedge_closed_form_on_gpu():
    H = from_lists(9, [list(range(9))], [4.0])
    x0c, x0b = start_block(H.n, H.m, 2, 3)
    got = run_pipeline(H, x0c, x0b, 3, torch.float64)
    assert int(got["rank"][0]) == 2
    assert np.isclose(got["R"][0], 0.25, rtol=1e-12)


def test_deterministic_bitwise():
    H, k, S = workload("grid64x32_m2300")
    x0c, x0b = start_block(H.n, H.m, 4, 7)
    for dtype in (torch.float64, torch.float32):
        a = run_pipeline(H, x0c, x0b, 5, dtype)
        b = run_pipeline(H, x0c, x0b, 5, dtype)
        assert np.array_equal(a["R"], b["R"]) and np.array_equal(a["argvec"], b["argvec"])


@pytest.mark.slow
def test_end_to_end_benchmark_size_netlist():
    """The 210,000-vertex, 200,000-hyperedge netlist (K = 160) in both forms
    against the FP64 oracle on the same instance."""
    H, k, S = workload("grid500x420_m200k")
    x0c, x0b = start_block(H.n, H.m, S, 2)
    ref = O.hyperedge_resistance(H.n, H.eptr, H.pins, H.w, x0c, x0b, k)
    for dtype in (torch.float64, torch.float32):
        got = run_pipeline(H, x0c, x0b, k, dtype)
        err = rel_errors(got["R"], ref["R"])
        assert err["max"] <= TOL[dtype], (dtype, err)
        assert kendall_tau(got["R"], ref["R"]) >= 0.999
        w_r = float((H.w * got["R"]).sum())
        assert 1.0 <= w_r <= 160 + 1e-6
