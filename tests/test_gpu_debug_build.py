"""The bounds-checked build (-DHEF_DEBUG=1, libhef_debug.so) computes what the
regular build computes, raises no false alarm on valid inputs, and reports a
pin planted outside [0, n) as HEF_ERR_BOUNDS instead of reading outside its
arrays.  The debug library runs in a child process that selects it through
HEF_LIBRARY.  The planted index is n (one record past the end), so even an
unchecked read of it would stay inside the Krylov workspace."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from netlists import start_block, workload
from netlists.synth import grid_netlist
from tests._gpu import rel_errors, run_pipeline

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEF_ERR_BOUNDS = -8

CHILD = r"""
import json, sys
sys.path.insert(0, ROOT_DIR)
import torch
import paper_2511_06600_gb300 as hef
from netlists import start_block, workload
from netlists.synth import grid_netlist
from tests._gpu import run_pipeline, to_dev

out = {"checks": int(hef.lib().hef_debug_checks())}
# valid inputs through the whole path: no status bit may be set (run_pipeline checks)
H, k, S = workload("grid64x32_m2300")
x0c, x0b = start_block(H.n, H.m, S, 0)
out["R_small"] = run_pipeline(H, x0c, x0b, k, torch.float64)["R"].tolist()
H2 = grid_netlist(200, 100, 21000, 7)  # n + m above the persistent form's threshold
y0c, y0b = start_block(H2.n, H2.m, 2, 0)
out["R_large"] = run_pipeline(H2, y0c, y0b, 10, torch.float32)["R"].tolist()
# a pin planted one past the end, in both Krylov forms
planted = []
for persistent in (1, 0):
    hef.set_krylov_persistent(persistent)
    t = to_dev(H2, y0c, y0b)
    inc = hef.build_incidence(H2.n, t["eptr"], t["pins"], t["w"])
    inc.check()
    inc.debug_set_pin(H2.P // 2, H2.n)
    hef.krylov_basis(inc, t["x0c"], t["x0b"], 10, torch.float32)
    try:
        inc.check()
        planted.append(0)
    except hef.HefError as e:
        planted.append(e.status)
hef.set_krylov_persistent(1)
out["planted"] = planted
print(json.dumps(out))
"""


def test_bounds_checked_build_agrees_and_reports_a_planted_index():
    from paper_2511_06600_gb300 import build
    path = build.build(debug=True)
    env = dict(os.environ, HEF_LIBRARY=path)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT_DIR", repr(ROOT))], env=env,
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["checks"] == 1
    # the regular build in this process, same inputs
    H, k, S = workload("grid64x32_m2300")
    x0c, x0b = start_block(H.n, H.m, S, 0)
    ref = run_pipeline(H, x0c, x0b, k, torch.float64)["R"]
    assert rel_errors(np.array(out["R_small"]), ref)["normwise"] <= 1e-12
    H2 = grid_netlist(200, 100, 21000, 7)
    y0c, y0b = start_block(H2.n, H2.m, 2, 0)
    ref2 = run_pipeline(H2, y0c, y0b, 10, torch.float32)["R"]
    assert rel_errors(np.array(out["R_large"]), ref2)["normwise"] <= 1e-5
    assert out["planted"] == [HEF_ERR_BOUNDS, HEF_ERR_BOUNDS]
