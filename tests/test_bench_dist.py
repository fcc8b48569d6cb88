"""Host logic of the multi-GPU benchmark line, on CPU with two gloo ranks:
the max-over-ranks time and the sum of the pins of all ranks (weak scaling:
each rank scores its own netlist, seed shifted by rank), and the reference
arm doing no work on ranks other than 0."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.getcwd())
import torch
import torch.distributed as dist
import bench
world, rank, _ = bench.dist_env()
dist.init_process_group("gloo", rank=rank, world_size=world)
cpu = torch.device("cpu")
H, k, S = bench.instance("grid64x32_m2300", rank)
t_max = bench.max_over_ranks(1.5 + rank, world, cpu)
p_all = bench.sum_over_ranks(H.P, world, cpu)
dist.barrier()
print(json.dumps({"rank": rank, "t_max": t_max, "p_all": p_all, "P": int(H.P),
                  "pins": H.pins[:32].tolist()}), flush=True)
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_max_time_and_total_pins():
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], cwd=ROOT, env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    assert all(o["t_max"] == 2.5 for o in outs)          # the slowest rank's time
    total = outs[0]["P"] + outs[1]["P"]
    assert all(o["p_all"] == total for o in outs)        # every rank's pins count
    assert outs[0]["pins"] != outs[1]["pins"]            # each rank has its own netlist


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2",
                                      "--steps", "1", "--warmup", "1"])
    bench.run_reference(bench.parse())
    assert capsys.readouterr().out == ""
