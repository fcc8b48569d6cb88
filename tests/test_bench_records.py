"""Host logic of the benchmark's roofline record: the committed DRAM-traffic
figures are reported only while the sources they were captured from still
hash to the recorded value, and every kernel in the record has a byte model
(the algorithmic bytes the roofline divides by)."""
import hashlib
import math
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from netlists import workload  # noqa: E402

RECORD = os.path.join(ROOT, "profiles", "dram_traffic_grid500x420_m200k_f32.txt")


def entries():
    out = []
    for line in open(RECORD):
        f = line.split()
        if len(f) == 4 and not line.startswith("#"):
            out.append((f[0], int(f[1]), f[2], f[3].split(",")))
    return out


def test_record_lines_are_well_formed():
    es = entries()
    assert "k_krylov_steps" in {e[0] for e in es}  # the dominant kernel of the step
    for name, nbytes, digest, files in es:
        assert nbytes > 0 and len(digest) == 64, name
        for f in files:
            assert os.path.exists(os.path.join(ROOT, f)), (name, f)


def test_traffic_reported_only_for_matching_sources(tmp_path, monkeypatch):
    es = entries()
    # the record as committed: a kernel is reported exactly when its sources
    # still hash to the recorded value
    for name, nbytes, digest, files in es:
        h = hashlib.sha256()
        for f in files:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        got = bench.recorded_traffic(name, "grid500x420_m200k", "f32")
        assert got == (nbytes if h.hexdigest() == digest else None), name
    # a copy of the tree where one source of the first kernel changed
    name, nbytes, digest, files = es[0]
    root = tmp_path / "tree"
    for f in files + ["profiles/dram_traffic_grid500x420_m200k_f32.txt"]:
        dst = root / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, f), dst)
    monkeypatch.setattr(bench, "ROOT", str(root))
    h = hashlib.sha256()
    for f in files:
        h.update((root / f).read_bytes())
    before = bench.recorded_traffic(name, "grid500x420_m200k", "f32")
    assert before == (nbytes if h.hexdigest() == digest else None)
    with open(root / files[0], "a") as fh:
        fh.write("\n// changed\n")
    assert bench.recorded_traffic(name, "grid500x420_m200k", "f32") is None
    assert bench.recorded_traffic("k_no_such_kernel", "grid500x420_m200k", "f32") is None
    assert bench.recorded_traffic(name, "no_such_workload", "f32") is None


def test_every_recorded_kernel_has_a_byte_model():
    H, k, S = workload("grid500x420_m200k")
    K = 2 * k * S
    for name, nbytes, _, _ in entries():
        bound, units = bench.kernel_model(name, H, K, S, k, 4)
        assert bound == "hbm" and math.isfinite(units) and units > 0, name
        # the cold-replay traffic stays within a small multiple of the model
        assert nbytes < 4 * units, (name, nbytes, units)
