"""hef_resistance_host (Algorithm 1 from host arrays, through the C ABI):
the scores equal the device-array path's bit for bit (same kernels, same
order), in both forms; repeated calls through the same page-locked buffers
(replayed as a CUDA graph from the second call on) score new contents;
a malformed hypergraph is reported, not scored."""
import numpy as np
import pytest
import torch

from netlists import start_block, workload
from tests._gpu import run_pipeline
from tests._hypergraphs import from_lists

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_host_call_equals_device_path(dtype):
    import paper_2511_06600_gb300 as h
    H, k, S = workload("grid64x32_m2300")
    x0c, x0b = start_block(H.n, H.m, 2, 3)
    ref = run_pipeline(H, x0c, x0b, k, dtype)
    R = h.resistance_host(H.n, torch.from_numpy(H.eptr), torch.from_numpy(H.pins),
                          torch.from_numpy(H.w), torch.from_numpy(x0c), torch.from_numpy(x0b),
                          k, dtype)
    assert np.array_equal(R.numpy(), ref["R"])


def test_host_call_reports_invalid_input():
    import paper_2511_06600_gb300 as h
    H = from_lists(4, [[0, 1], [1, 7]])  # pin 7 is outside [0, 4)
    x0c, x0b = start_block(H.n, H.m, 1, 0)
    with pytest.raises(h.HefError) as ei:
        h.resistance_host(H.n, torch.from_numpy(H.eptr), torch.from_numpy(H.pins),
                          torch.from_numpy(H.w), torch.from_numpy(x0c), torch.from_numpy(x0b),
                          2, torch.float64)
    assert ei.value.status == -7


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_repeated_host_calls_through_pinned_buffers_score_new_contents(dtype):
    """Calls 1 (eager), 2 (captured) and 3-4 (replayed) through the same
    page-locked buffers, each with other weights and starts of the same
    sizes: every call equals the device-array path on its own inputs."""
    import paper_2511_06600_gb300 as h
    H, k, S = workload("grid64x32_m2300")
    eptr = torch.from_numpy(H.eptr).pin_memory()
    pins = torch.from_numpy(H.pins).pin_memory()
    w = torch.empty(H.m, dtype=torch.float64).pin_memory()
    x0c = torch.empty(H.n, 2, dtype=torch.float64).pin_memory()
    x0b = torch.empty(H.n + H.m, 2, dtype=torch.float64).pin_memory()
    R = torch.empty(H.m, dtype=torch.float64).pin_memory()
    ws = h.resistance_host_workspace(H.n, H.m, H.P, k, 2, dtype)
    rng = np.random.default_rng(5)
    for call in range(4):
        wv = np.exp(rng.uniform(np.log(0.5), np.log(2.0), H.m))
        a, b = start_block(H.n, H.m, 2, 10 + call)
        w.copy_(torch.from_numpy(wv))
        x0c.copy_(torch.from_numpy(a))
        x0b.copy_(torch.from_numpy(b))
        h.resistance_host(H.n, eptr, pins, w, x0c, x0b, k, dtype, R_out=R, workspace=ws)
        ref = _device_scores(H, wv, a, b, k, dtype)
        assert np.array_equal(R.numpy(), ref), call


def _device_scores(H, wv, x0c, x0b, k, dtype):
    import paper_2511_06600_gb300 as h
    dev = torch.device("cuda:0")
    out = h.hyperedge_resistance(H.n, torch.from_numpy(H.eptr).to(dev),
                                 torch.from_numpy(H.pins).to(dev), torch.from_numpy(wv).to(dev),
                                 torch.from_numpy(x0c).to(dev), torch.from_numpy(x0b).to(dev), k,
                                 dtype)
    torch.cuda.synchronize()
    return out["R"].cpu().numpy()
