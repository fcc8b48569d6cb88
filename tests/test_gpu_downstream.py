"""Consumers of the scores on the GPU (hef_sort_resistance, hef_coarsen_level
through the C ABI) against the CPU oracle (oracle/hef_downstream.py), bit for
bit, when both are fed identical inputs: the GPU's own scores R, basis Q and
Q_H.  Covers Algorithm 1 step 6, Eq. R_W_update, the greedy contraction of
Algorithm 2 step 5, the local clustering of steps 7-10 and the coarse
hypergraph of step 6, on small and mid-size netlists (with ties, 1-pin
hyperedges and non-zero supernode weights), a three-level sweep, and the
full 210k-vertex netlist (the local clustering sampled there)."""
import numpy as np
import pytest
import torch

from netlists import start_block, workload
from netlists.synth import grid_netlist
from oracle import hef_downstream as D
from tests._gpu import DEV, to_dev
from tests._hypergraphs import from_lists, random_hypergraph

pytestmark = pytest.mark.gpu


def hef():
    import paper_2511_06600_gb300 as m
    return m


def scores_on_gpu(H, k, S, dtype, seed=0):
    h = hef()
    x0c, x0b = start_block(H.n, H.m, S, seed)
    t = to_dev(H, x0c, x0b)
    inc = h.build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    K = 2 * k * S
    V = h.krylov_basis(inc, t["x0c"], t["x0b"], k, dtype)
    Q, _, _ = h.orthonormalize(V, K)
    sc = h.edge_resistance(inc, Q, K)
    inc.check()
    return t, inc, Q, K, sc


def gpu_level(t, inc, R, eta, Q, K, QH, delta=-1.0, q=0.5):
    h = hef()
    out = h.coarsen_level(inc, t["eptr"], t["pins"], t["w"], R, eta, Q, K, QH, delta=delta,
                          quantile=q)
    nc, nf, mc, pc = h.level_sizes(out)
    n, m = inc.n, inc.m
    got = {key: out[key].cpu().numpy() for key in out if key != "_keep"}
    got.update(nc=nc, nf=nf, mc=mc, pc=pc)
    got["R_upd"], got["order"], got["emap"] = got["R_upd"][:m], got["order"][:m], got["emap"][:mc]
    for key in ("owner", "cluster", "target", "dist", "final_cluster"):
        got[key] = got[key][:n]
    got["eta_out"] = got["eta_out"][:nf]
    got["ceptr"], got["cpins"], got["cw"] = got["ceptr"][:mc + 1], got["cpins"][:pc], got["cw"][:mc]
    return got


def assert_level_equal(got, want):
    """Every output of the level, compared exactly (FP64 values bitwise)."""
    assert np.array_equal(got["R_upd"], want["R_upd"])
    assert np.array_equal(got["order"], want["order"])
    assert got["delta"][0] == want["delta"]
    assert np.array_equal(got["owner"], want["owner"])
    assert np.array_equal(got["cluster"], want["cluster"]) and got["nc"] == want["nc"]
    assert np.array_equal(got["target"], want["target"])
    assert np.array_equal(got["dist"], want["dist"])
    assert np.array_equal(got["final_cluster"], want["final"]) and got["nf"] == want["nf"]
    assert np.array_equal(got["eta_out"], want["eta"])
    assert np.array_equal(got["ceptr"], want["eptr"])
    assert np.array_equal(got["cpins"], want["pins"])
    assert np.array_equal(got["cw"], want["w"])
    assert np.array_equal(got["emap"], want["emap"])


def oracle_level(H, R, Q, QH, eta, delta=None, q=0.5):
    return D.level(H.n, H.eptr, H.pins, H.w, R, Q, QH, eta, delta=delta, q=q)


def test_sort_matches_oracle_with_ties_and_zeros():
    rng = np.random.default_rng(3)
    for m in (0, 1, 7, 5000, 70001):
        R = rng.integers(0, 5, size=m).astype(np.float64) / 4  # ties and zeros
        mask = rng.uniform(size=m) < 0.3
        R[mask] = rng.uniform(size=int(mask.sum()))
        order = hef().sort_resistance(torch.from_numpy(R).to(DEV)).cpu().numpy()
        assert order.tolist() == D.sort_order(R).tolist(), m


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("q", [0.5, 0.8])
def test_level_bit_exact_small_netlist(dtype, q):
    H, k, S = workload("grid64x32_m2300")
    t, inc, Q, K, sc = scores_on_gpu(H, k, 2, dtype)
    R = sc["R"].cpu().numpy()
    Qh = Q[:, :K].cpu().numpy()
    QH = sc["QH"].cpu().numpy()
    got = gpu_level(t, inc, sc["R"], None, Q, K, sc["QH"], q=q)
    assert_level_equal(got, oracle_level(H, R, Qh, QH, np.zeros(H.n), q=q))


def test_level_bit_exact_ties_one_pin_edges_and_weights():
    # random hypergraph with 1-pin hyperedges and ties in R, a given delta,
    # non-zero supernode weights from a previous level
    rng = np.random.default_rng(11)
    base = random_hypergraph(300, 420, 7, 5, weights=True, min_size=1)
    H = base
    t = to_dev(H)
    inc = hef().build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    R = rng.integers(1, 6, size=H.m).astype(np.float64) / 8
    eta = rng.uniform(0, 1, size=H.n) * (rng.uniform(size=H.n) < 0.4)
    K = 12
    Qh = rng.standard_normal((H.n, K)).astype(np.float32)
    QH = rng.uniform(0.5, 2, size=K)
    QH[3] = 0.0
    Qd = torch.zeros(H.n, 16, dtype=torch.float32)
    Qd[:, :K] = torch.from_numpy(Qh)
    got = gpu_level(t, inc, torch.from_numpy(R).to(DEV), torch.from_numpy(eta).to(DEV),
                    Qd.to(DEV), K, torch.from_numpy(QH).to(DEV), delta=0.5)
    assert_level_equal(got, oracle_level(H, R, Qh, QH, eta, delta=0.5))


def test_level_degenerate_inputs():
    h = hef()
    # no hyperedge qualifies (delta = 0); an isolated vertex; an empty hyperedge
    H = from_lists(6, [[0, 1], [], [2], [3, 4, 1]], [1.0, 1.0, 2.0, 0.5])
    t = to_dev(H)
    inc = h.build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    R = np.array([0.5, 0.0, 0.0, 0.25])
    K = 4
    Qh = np.arange(H.n * K, dtype=np.float64).reshape(H.n, K) / 7
    QH = np.ones(K)
    Qd = torch.from_numpy(Qh).to(DEV)
    for delta in (0.0, 10.0):
        got = gpu_level(t, inc, torch.from_numpy(R).to(DEV), None, Qd, K,
                        torch.from_numpy(QH).to(DEV), delta=delta)
        assert_level_equal(got, oracle_level(H, R, Qh, QH, np.zeros(H.n), delta=delta))
    # without a basis: no local clustering
    out = h.coarsen_level(inc, t["eptr"], t["pins"], t["w"], torch.from_numpy(R).to(DEV),
                          delta=10.0)
    nc, nf, mc, pc = h.level_sizes(out)
    assert (out["target"][:H.n] == -1).all() and nf == nc


def test_three_level_sweep_each_level_bit_exact():
    h = hef()
    H = grid_netlist(100, 80, 8400, 31, size_law="pareto400", radius_law="sqrt",
                     long_range=0.02)
    k, S = 6, 2

    def starts(level, n, m):
        x0c, x0b = start_block(n, m, S, 100 + level)
        return torch.from_numpy(x0c).to(DEV), torch.from_numpy(x0b).to(DEV)

    t = to_dev(H)
    levels, of_orig = h.multilevel(H.n, t["eptr"], t["pins"], t["w"], starts, k, 3,
                                   torch.float32, quantile=0.5)
    assert len(levels) == 3
    eta = np.zeros(H.n)
    for lv in levels:
        from netlists import Netlist
        Hl = Netlist(n=lv["n"], eptr=lv["eptr"].cpu().numpy(), pins=lv["pins"].cpu().numpy(),
                     w=lv["w"].cpu().numpy())
        want = oracle_level(Hl, lv["R"].cpu().numpy(), lv["Q"][:, :lv["K"]].cpu().numpy(),
                            lv["QH"].cpu().numpy(), eta)
        lo = lv["level"]
        assert lv["nf"] == want["nf"] and lv["m_next"] == len(want["emap"])
        assert np.array_equal(lo["final_cluster"][:lv["n"]].cpu().numpy(), want["final"])
        assert np.array_equal(lo["eta_out"][:lv["nf"]].cpu().numpy(), want["eta"])
        assert np.array_equal(lo["cpins"][:lv["P_next"]].cpu().numpy(), want["pins"])
        eta = want["eta"]
        assert lv["nf"] < lv["n"]  # every level coarsens
    assert int(of_orig.max()) + 1 == levels[-1]["nf"]


def test_level_full_size_netlist():
    """grid500x420_m200k (FP32 scores): Eq. R_W_update, the sort, delta, the
    contraction and the supernodes exactly; the local clustering's choice on
    400 sampled isolated vertices; the final clusters, weights and coarse
    hypergraph exactly, given the GPU's choices."""
    H, k, S = workload("grid500x420_m200k")
    t, inc, Q, K, sc = scores_on_gpu(H, k, S, torch.float32)
    got = gpu_level(t, inc, sc["R"], None, Q, K, sc["QH"], q=0.5)
    R = sc["R"].cpu().numpy()
    eta = np.zeros(H.n)
    Ru = D.update_resistance(H.eptr, H.pins, R, eta)
    assert np.array_equal(got["R_upd"], Ru)
    order = np.lexsort((np.arange(H.m), Ru))
    assert np.array_equal(got["order"], order)
    assert D.sort_order(Ru[:2000]).tolist() == np.lexsort((np.arange(2000), Ru[:2000])).tolist()
    delta = D.quantile_threshold(Ru, np.diff(H.eptr), 0.5)
    assert got["delta"][0] == delta
    owner, contracted = D.contract(H.n, H.eptr, H.pins, order, Ru, delta)
    assert np.array_equal(got["owner"], owner)
    cluster, nc, eta_next, formed_by = D.clusters(H.n, H.eptr, H.pins, owner, contracted, Ru, eta)
    assert np.array_equal(got["cluster"], cluster) and got["nc"] == nc
    # sampled local-clustering choices, computed one by one by the oracle
    vptr, vedge = D.vertex_incidence(H.n, H.eptr, H.pins)
    Qh = Q[:, :K].cpu().numpy()
    QH = sc["QH"].cpu().numpy()
    seeds = np.flatnonzero(owner < 0)
    rng = np.random.default_rng(0)
    cache = {}
    for p in rng.choice(seeds, size=min(400, len(seeds)), replace=False):
        c, d = D.seed_choice(int(p), H.eptr, H.pins, vptr, vedge, cluster, formed_by, Qh, QH, cache)
        assert got["target"][p] == c and got["dist"][p] == d, p
    assert (got["target"][owner >= 0] == -1).all()
    # steps 7-9 from the GPU's choices
    eta2 = eta_next.copy()
    for p in np.flatnonzero(got["target"] >= 0):
        eta2[got["target"][p]] += float(eta[p]) + float(got["dist"][p])
    final, nf, eta_f = D.final_clusters(H.n, cluster, got["target"], eta2)
    assert np.array_equal(got["final_cluster"], final) and got["nf"] == nf
    assert np.array_equal(got["eta_out"], eta_f)
    ce, cp, cw, emap = D.coarsen(H.eptr, H.pins, H.w, final)
    assert np.array_equal(got["ceptr"], ce) and np.array_equal(got["cpins"], cp)
    assert np.array_equal(got["cw"], cw) and np.array_equal(got["emap"], emap)
