"""The BF16 storage form (HEF_BF16) through the C ABI: the archived basis is
exactly the FP32 form's chain values rounded to BF16; CholQR2 on the tensor
cores leaves its columns orthonormal to BF16 precision; scoring a BF16 basis
equals scoring the same values widened to FP32; and the scores' error
against the FP64 oracle is measured and bounded as the BF16 rounding allows
(it does not meet the reduced forms' 2e-3; see test_bf16_storage_oracle)."""
import numpy as np
import pytest
import torch

from netlists import start_block, workload
from netlists.synth import grid_netlist
from oracle import hef_oracle as O
from tests._gpu import DEV, kendall_tau, rel_errors, to_dev

pytestmark = pytest.mark.gpu


def hef():
    import paper_2511_06600_gb300 as m
    return m


def _setup(H, k, S, seed=1):
    h = hef()
    x0c, x0b = start_block(H.n, H.m, S, seed)
    t = to_dev(H, x0c, x0b)
    inc = h.build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    return h, t, inc, x0c, x0b


@pytest.mark.parametrize("persistent", [1, 0])
def test_bf16_archive_is_rounded_fp32_archive(persistent):
    H = grid_netlist(200, 100, 21000, 9)  # above the persistent form's size
    k, S = 6, 4
    h, t, inc, _, _ = _setup(H, k, S)
    h.set_krylov_persistent(persistent)
    try:
        V32 = h.krylov_basis(inc, t["x0c"], t["x0b"], k, torch.float32)
        Vbf = h.krylov_basis(inc, t["x0c"], t["x0b"], k, torch.bfloat16)
    finally:
        h.set_krylov_persistent(1)
    K = 2 * k * S
    assert torch.equal(Vbf[:, :K], V32[:, :K].to(torch.bfloat16))


def test_bf16_orthonormal_to_bf16_precision_and_scoring_matches_fp32_kernels():
    H, k, S = workload("grid64x32_m2300")
    S = 4
    h, t, inc, _, _ = _setup(H, k, S)
    K = 2 * k * S
    V = h.krylov_basis(inc, t["x0c"], t["x0b"], k, torch.bfloat16)
    Q, _, rank = h.orthonormalize(V, K)
    assert int(rank.item()) == K
    Qd = Q[:, :K].double()
    Qc = Qd - Qd.mean(dim=0)
    G = Qc.T @ Qc
    assert (G - torch.eye(K, dtype=torch.float64, device=DEV)).abs().max() < 3e-2
    assert Qd.mean(dim=0).abs().max() < 1e-3
    # scoring the BF16 basis = scoring its values widened to FP32 (FP32 arithmetic)
    a = h.edge_resistance(inc, Q, K)
    Q32 = torch.zeros(H.n, h.padded_ld(K, torch.float32), dtype=torch.float32, device=DEV)
    Q32[:, :K] = Q[:, :K].float()
    b = h.edge_resistance(inc, Q32, K)
    ra, rb = a["R"].cpu().numpy(), b["R"].cpu().numpy()
    assert np.allclose(a["QH"].cpu().numpy(), b["QH"].cpu().numpy(), rtol=1e-6, atol=0)
    assert np.allclose(ra, rb, rtol=1e-5, atol=0)
    agree = (a["argvec"] == b["argvec"]).float().mean().item()
    assert agree > 0.999, agree


def test_bf16_scores_against_oracle():
    H = grid_netlist(100, 80, 8400, 3)
    k, S = 12, 4
    h, t, inc, x0c, x0b = _setup(H, k, S, seed=3)
    out = h.hyperedge_resistance(H.n, t["eptr"], t["pins"], t["w"], t["x0c"], t["x0b"], k,
                                 torch.bfloat16)
    R = out["R"].cpu().numpy()
    ref = O.hyperedge_resistance(H.n, H.eptr, H.pins, H.w, x0c, x0b, k)["R"]
    err = rel_errors(R, ref)
    tau = kendall_tau(R, ref)
    # what BF16 storage allows (the oracle experiment gives max 1.5e-2,
    # p99 9e-3, normwise 2.3e-3 on this netlist)
    assert err["normwise"] < 1e-2 and err["p99"] < 3e-2 and tau > 0.99, (err, tau)
    # the EMBED scoring and the downstream level accept the BF16 basis
    Q, K = out["Q"], 2 * k * S
    emb = h.edge_resistance(out["incidence"], Q, K, reduce=h.HEF_REDUCE_EMBED)
    assert (emb["R"] <= out["R"] * (1 + 1e-5)).all()
    lo = h.coarsen_level(out["incidence"], t["eptr"], t["pins"], t["w"], out["R"], None, Q, K,
                         out["QH"])
    nc, nf, mc, pc = h.level_sizes(lo)
    assert 0 < nf < H.n
