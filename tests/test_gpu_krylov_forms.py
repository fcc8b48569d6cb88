"""The two launch forms of the Krylov calls (one persistent launch with
bounded grid barriers, or three launches per step) give the same scores, and
a barrier wait that cannot complete is reported through the incidence's
status word (HEF_ERR_TIMEOUT) without hanging the GPU; the context stays
usable afterwards."""
import numpy as np
import pytest
import torch

from netlists import start_block, workload
from netlists.synth import grid_netlist
from oracle import hef_oracle as O
from tests._gpu import DEV, rel_errors, run_pipeline, to_dev

pytestmark = pytest.mark.gpu

HEF_ERR_TIMEOUT = -5


def hef():
    import paper_2511_06600_gb300 as m
    return m


@pytest.fixture(autouse=True)
def restore_default():
    yield
    hef().set_krylov_persistent(1)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
def test_persistent_and_per_step_forms_agree(dtype, tol):
    # n + m = 41,000 rows: above the size from which the persistent form runs
    H = grid_netlist(200, 100, 21000, 7)
    k = 10
    x0c, x0b = start_block(H.n, H.m, 2, 0)
    hef().set_krylov_persistent(1)
    a = run_pipeline(H, x0c, x0b, k, dtype)
    hef().set_krylov_persistent(0)
    b = run_pipeline(H, x0c, x0b, k, dtype)
    err = rel_errors(a["R"], b["R"])
    assert err["normwise"] <= tol, err
    ref = O.hyperedge_resistance(H.n, H.eptr, H.pins, H.w, x0c, x0b, k)["R"]
    bound = 1e-9 if dtype == torch.float64 else 2e-3
    assert rel_errors(a["R"], ref)["max"] <= bound


def test_barrier_timeout_is_reported_and_recoverable():
    h = hef()
    H = grid_netlist(300, 300, 95000, 21)  # 2n + m > twice the resident threads
    k, S = 4, 1
    x0c, x0b = start_block(H.n, H.m, S, 1)
    t = to_dev(H, x0c, x0b)
    h.set_krylov_persistent(2)
    out = h.hyperedge_resistance(H.n, t["eptr"], t["pins"], t["w"], t["x0c"], t["x0b"], k,
                                 torch.float64, check=False)
    torch.cuda.synchronize()
    with pytest.raises(h.HefError) as exc:
        out["incidence"].check()
    assert exc.value.status == HEF_ERR_TIMEOUT
    # the GPU context is intact: the same inputs score normally afterwards
    h.set_krylov_persistent(1)
    good = h.hyperedge_resistance(H.n, t["eptr"], t["pins"], t["w"], t["x0c"], t["x0b"], k,
                                  torch.float64)
    R = good["R"].cpu().numpy()
    assert np.isfinite(R).all() and R.max() > 0
