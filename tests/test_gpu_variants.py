"""Variants of Algorithm 1 on the GPU (through the C ABI) against the oracle:

* the single-expansion Krylov pool (hef_krylov_basis_ops; HEF_OPS_STAR is the
  earlier HyperEF pool that Section III-A.3 contrasts with the mixed one):
  its columns are exactly the matching columns of the mixed basis, and its
  scores match the oracle's star-only scores at the FP64 / FP32 tolerances;
* EMBED scoring (HEF_REDUCE_EMBED, reading A7's alternative): the farthest
  pin pair, the arg-max column and the pair's routing equal the oracle's
  exactly (the pair is decided in FP64 with the oracle's summation order),
  the scores within the rounding of Q_H's sum."""
import numpy as np
import pytest
import torch

from netlists import start_block, workload
from netlists.synth import grid_netlist
from oracle import hef_oracle as O
from tests._gpu import DEV, rel_errors, to_dev

pytestmark = pytest.mark.gpu


def hef():
    import paper_2511_06600_gb300 as m
    return m


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("ops", ["star", "clique"])
def test_single_expansion_pool_columns_and_scores(dtype, ops):
    h = hef()
    H, k, S = workload("grid64x32_m2300")
    S = 2
    x0c, x0b = start_block(H.n, H.m, S, 4)
    t = to_dev(H, x0c, x0b)
    inc = h.build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    code = h.HEF_OPS_STAR if ops == "star" else h.HEF_OPS_CLIQUE
    op = 1 if ops == "star" else 0
    Vboth = h.krylov_basis(inc, t["x0c"], t["x0b"], k, dtype)
    Vone = h.krylov_basis(inc, t["x0c"], t["x0b"], k, dtype, ops=code)
    torch.cuda.synchronize()
    Kb = k * S
    for j in range(k):
        for s in range(S):
            assert torch.equal(Vone[:, j * S + s], Vboth[:, j * 2 * S + op * S + s])
    got = h.hyperedge_resistance(H.n, t["eptr"], t["pins"], t["w"], t["x0c"], t["x0b"], k, dtype,
                                 ops=code)
    R = got["R"].cpu().numpy()
    ref = O.hyperedge_resistance(H.n, H.eptr, H.pins, H.w, x0c, x0b, k, ops=ops)["R"]
    tol = 1e-9 if dtype == torch.float64 else 2e-3
    err = rel_errors(R, ref)
    assert (err["max"] if dtype == torch.float64 else err["normwise"]) <= tol, err
    assert got["Q"].shape[1] == Kb


def _embed_case(H, k, S, dtype):
    h = hef()
    x0c, x0b = start_block(H.n, H.m, S, 6)
    t = to_dev(H, x0c, x0b)
    inc = h.build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    K = 2 * k * S
    V = h.krylov_basis(inc, t["x0c"], t["x0b"], k, dtype)
    Q, _, _ = h.orthonormalize(V, K)
    plain = h.edge_resistance(inc, Q, K)
    emb = h.edge_resistance(inc, Q, K, reduce=h.HEF_REDUCE_EMBED)
    inc.check()
    got = {key: v.cpu().numpy() for key, v in emb.items()}
    Qh = Q[:, :K].cpu().numpy()
    want = O.edge_resistance_embed(Qh, H.eptr, H.pins, H.w)
    assert np.array_equal(got["QH"], plain["QH"].cpu().numpy())
    assert np.array_equal(got["argvec"], want["argvec"])
    assert np.array_equal(got["pmax"], want["pmax"])
    assert np.array_equal(got["pmin"], want["pmin"])
    # R_e is exactly (Q[p,i*] - Q[q,i*])^2 / Q_H[i*] with the call's own Q_H,
    # which matches the oracle's to the form's rounding
    ok = got["argvec"] >= 0
    i = got["argvec"][ok]
    diff = Qh[got["pmax"][ok], i].astype(np.float64) - Qh[got["pmin"][ok], i].astype(np.float64)
    assert np.array_equal(got["R"][ok], diff * diff / got["QH"][i])
    assert (got["R"][~ok] == 0).all()
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    assert np.allclose(got["QH"], want["QH"], rtol=tol, atol=0)
    assert np.allclose(got["R"], want["R"], rtol=10 * tol, atol=0)
    # EMBED never exceeds the max-min scores (any pair spans at most the
    # spread); the FP32 form rounds the spread to FP32, EMBED's difference is
    # exact, so there the bound holds to FP32 rounding
    slack = 1e-12 if dtype == torch.float64 else 4e-6
    assert (got["R"] <= plain["R"].cpu().numpy() * (1 + slack)).all()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_embed_small_netlist(dtype):
    H, k, S = workload("grid64x32_m2300")
    _embed_case(H, k, 2, dtype)


def test_embed_pareto_netlist_with_large_hyperedges():
    H = grid_netlist(120, 90, 10000, 12, size_law="pareto400", radius_law="sqrt",
                     long_range=0.02)
    assert int(H.sizes().max()) > 100
    _embed_case(H, 5, 2, torch.float32)
