"""The precision form at its own scale (1200 x 1000 grid, 1.3M nets, k = 24,
S = 8, K = 384, FP32 basis, the launch configuration the benchmark times):
properties that hold at any size on the full instance, and element-wise
agreement with the FP64 oracle on the induced 400 x 250 window."""
import numpy as np
import pytest
import torch

from netlists import start_block, window_subhypergraph, workload
from oracle import hef_oracle as O
from tests._gpu import DEV, kendall_tau, rel_errors, to_dev

pytestmark = pytest.mark.gpu


def hef():
    import paper_2511_06600_gb300 as m
    return m


@pytest.mark.slow
def test_precision_form_full_size_and_window_vs_oracle():
    H, k, S = workload("grid1200x1000_m1300k")
    K = 2 * k * S
    x0c, x0b = start_block(H.n, H.m, S, 3)
    t = to_dev(H, x0c, x0b)
    pipe = hef().Pipeline(H.n, H.m, H.P, k, S, torch.float32, device=DEV)
    out = pipe.run(t["eptr"], t["pins"], t["w"], t["x0c"], t["x0b"])
    torch.cuda.synchronize()
    pipe.check()
    R = out["R"].cpu().numpy()
    rank = int(pipe.rank.item())
    assert rank == K
    assert np.isfinite(R).all() and (R >= 0).all()
    # sum_e w_e r_e(chi) = 1 for every column (definition of Q_H), hence
    # 1 <= sum_e w_e R_e <= rank for the max over columns
    s = float(H.w @ R)
    assert 1.0 - 1e-4 <= s <= rank * (1 + 1e-4), s
    assert (out["QH"].cpu().numpy() > 0).all()
    # element-wise on the 100k-cell window
    Hs = window_subhypergraph(H, 0, 400, 0, 250)
    xs, xb = start_block(Hs.n, Hs.m, S, 3)
    tw = to_dev(Hs, xs, xb)
    got = hef().hyperedge_resistance(Hs.n, tw["eptr"], tw["pins"], tw["w"], tw["x0c"], tw["x0b"],
                                     k, torch.float32)["R"].cpu().numpy()
    ref = O.hyperedge_resistance(Hs.n, Hs.eptr, Hs.pins, Hs.w, xs, xb, k)["R"]
    err = rel_errors(got, ref)
    assert err["normwise"] <= 2e-3 and err["p99"] <= 2e-3, err
    assert kendall_tau(got, ref) >= 0.999
