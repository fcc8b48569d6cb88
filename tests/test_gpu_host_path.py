"""hef_resistance_host (Algorithm 1 from host arrays, through the C ABI):
the scores equal the device-array path's bit for bit (same kernels, same
order), in both forms; a malformed hypergraph is reported, not scored."""
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
