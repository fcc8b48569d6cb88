"""hef_edge_resistance_noalloc: scoring for callers that cannot give the
library device memory (no allocator of their own, or a GPU whose memory a
pool already owns).  Its scratch is a fixed array inside the library, so two
calls in a row must both reproduce the regular entry point's scores.  This
file is collected last on purpose."""
import numpy as np
import pytest
import torch

from netlists import start_block, workload
from tests._gpu import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_scores_match_workspace_call_twice(dtype):
    import paper_2511_06600_gb300 as hef
    H, k, S = workload("grid64x32_m2300")
    x0c, x0b = start_block(H.n, H.m, 2, 5)
    t = to_dev(H, x0c, x0b)
    inc = hef.build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    K = 2 * k * 2
    V = hef.krylov_basis(inc, t["x0c"], t["x0b"], k, dtype)
    Q, _, _ = hef.orthonormalize(V, K)
    ref = hef.edge_resistance(inc, Q, K)
    inc.check()
    ref = {key: v.cpu().numpy() for key, v in ref.items()}
    for _ in range(2):
        got = hef.edge_resistance_noalloc(inc, Q, K)
        torch.cuda.synchronize()
        got = {key: v.cpu().numpy() for key, v in got.items()}
        assert np.allclose(got["QH"], ref["QH"], rtol=1e-12, atol=0)
        assert np.allclose(got["R"], ref["R"], rtol=1e-12, atol=0)
        assert np.array_equal(got["argvec"], ref["argvec"])
        assert np.array_equal(got["pmax"], ref["pmax"])
        assert np.array_equal(got["pmin"], ref["pmin"])


def test_noalloc_rejects_oversized_K():
    import paper_2511_06600_gb300 as hef
    H, _, _ = workload("grid64x32_m2300")
    t = to_dev(H)
    inc = hef.build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    Q = torch.zeros(H.n, 520, dtype=torch.float32, device="cuda:0")
    with pytest.raises(hef.HefError) as ei:
        hef.edge_resistance_noalloc(inc, Q, 513)
    assert ei.value.status == -6


@pytest.mark.parametrize("K,dtype", [(384, torch.float32), (512, torch.float32),
                                     (512, torch.float64)])
def test_noalloc_large_K_pareto_netlist_matches_workspace_call(K, dtype):
    """Large K takes the capped per-CTA partials; the Pareto tail gives
    hyperedges of more than 64 pins, which the large-hyperedge kernels score.
    Any basis is a valid input to the scoring, so Q is a seeded random matrix."""
    import paper_2511_06600_gb300 as hef
    from netlists.synth import grid_netlist
    H = grid_netlist(120, 80, 9000, seed=11, size_law="pareto400", radius_law="sqrt",
                     long_range=0.02)
    assert int(H.sizes().max()) > 64
    t = to_dev(H)
    inc = hef.build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    g = torch.Generator(device="cpu").manual_seed(K)
    ld = hef.padded_ld(K, dtype)
    Q = torch.zeros(H.n, ld, dtype=dtype)
    Q[:, :K] = torch.randn(H.n, K, generator=g, dtype=torch.float64).to(dtype)
    Q = Q.to("cuda:0")
    ref = hef.edge_resistance(inc, Q, K)
    inc.check()
    ref = {key: v.cpu().numpy() for key, v in ref.items()}
    for _ in range(2):
        got = hef.edge_resistance_noalloc(inc, Q, K)
        torch.cuda.synchronize()
        got = {key: v.cpu().numpy() for key, v in got.items()}
        assert np.allclose(got["QH"], ref["QH"], rtol=1e-12, atol=0)
        assert np.allclose(got["R"], ref["R"], rtol=1e-12, atol=0)
        assert np.array_equal(got["argvec"], ref["argvec"])
        assert np.array_equal(got["pmax"], ref["pmax"])
        assert np.array_equal(got["pmin"], ref["pmin"])
