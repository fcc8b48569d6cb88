#!/usr/bin/env python
"""Benchmark of hyperedge effective-resistance estimation (Algorithm 1) on GB300.

One step = the whole hot path on one synthetic netlist: incidence build,
Krylov basis (k steps of both expansions), CholQR2, scoring (two passes).
Default workload: 500x420 grid (n = 210,000), 200,000 nets (80 % 2-3 pins,
Pareto(2.2) tail capped at 400, 2 % long-range pins), k = 20 per expansion,
S = 4 starts, K = 160 basis vectors, FP32 form (FP64 Cholesky and Q_H); the
plain FP64 form is timed beside it for the speedup.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead, on a bounded window of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from netlists import start_block, window_subhypergraph, workload  # noqa: E402

METRIC = "pins/s of Krylov resistance scoring; HBM GB/s; speedup vs FP64 plain at tol"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grid500x420_m200k")
    ap.add_argument("--form", default="f32", choices=["f32", "f64"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-backward", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-precision-oracle", action="store_true")
    ap.add_argument("--batched-graphs", type=int, default=64)
    ap.add_argument("--backward-workload", default="grid500x400_m210k_logw")
    return ap.parse_args()


# ---------------------------------------------------------------- helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, world, device):
    """Largest x over the ranks (all-reduce MAX: NCCL on GPUs, gloo on CPU)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world, device):
    """Sum of x over the ranks (all-reduce SUM)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def instance(name, rank):
    """The rank's netlist: the named workload, seed shifted per rank (each
    rank scores its own netlist: weak scaling)."""
    from netlists.synth import WORKLOADS, grid_netlist
    cfg = dict(WORKLOADS[name])
    k, S = cfg.pop("k"), cfg.pop("S")
    cfg["seed"] = cfg["seed"] + 1000 * rank
    H = grid_netlist(name=name, **cfg)
    return H, k, S


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # start timing only once the sampler is producing rows
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0:
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def recorded_traffic(kernel, workload, form):
    """DRAM bytes per launch of `kernel` from the committed ncu record for this
    workload and form, or None when there is none or the kernel's sources
    changed after the capture (their sha256 no longer matches)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"dram_traffic_{workload}_{form}.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if len(f) != 4 or f[0] != kernel:
            continue
        h = hashlib.sha256()
        for src in f[3].split(","):
            p = os.path.join(ROOT, src)
            if not os.path.exists(p):
                return None
            h.update(open(p, "rb").read())
        return int(f[1]) if h.hexdigest() == f[2] else None
    return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured", d.get("sm_max_mhz", 2070.0)
    return 6800.0, "fallback", 2070.0


def kernel_model(name, H, K, S, k, esz):
    """Algorithmic (compulsory, cache-perfect) bytes or flops of one launch of
    `name`: ('hbm', bytes) or ('alu', flops)."""
    n, m, P = H.n, H.m, H.P
    if name == "k_gram":
        return "alu", float(n) * K * (K + 1)          # K(K+1)/2 dots of length n
    if name == "k_apply":
        return "alu", float(n) * K * (K + 1)          # triangular V R^-1
    if name == "k_gram_tc":       # V read once (plus the ones column), FP64 partials of G
        Kq = (K + 16) // 16 * 16
        return "hbm", float(n) * K * esz + 152 * Kq * Kq * 8.0 / 2
    if name == "k_apply_tc":      # V read and written in place
        return "hbm", 2.0 * n * K * esz
    if name == "k_score_pass1":   # Q once, the pin lists, offsets, weights; spreads written
        return "hbm", n * K * esz + 4.0 * P + 4.0 * (m + 1) + 8.0 * m + float(m) * K * esz
    if name == "k_score_ratio":   # spreads read; one column of Q per hyperedge's pins; outputs
        return "hbm", float(m) * K * esz + 4.0 * (m + 1) + 4.0 * m + 4.0 * P + esz * P + 20.0 * m
    if name == "k_score_pass2":
        return "hbm", n * K * esz + 4.0 * P + 4.0 * (m + 1) + 8.0 * m + 4.0 * m + 20.0 * m
    # Krylov passes: vertex records [x_c | x_b] (2S values), star hyperedge
    # rows (S values), edge records [wh s | z x_b] (2S values); the per-edge
    # and per-vertex scalars are read in the basis type (esz bytes)
    if name == "k_edge_pass":   # pin lists; vertex records once; own star rows (x_{j-1}, x_{j-2}); Ye, Er written
        return "hbm", 4.0 * P + 4.0 * (m + 1) + 3.0 * esz * m + esz * S * (2 * n + 5 * m)
    if name == "k_node_pass":   # incidence; own records (x_{j-1}, x_{j-2}); Er once; Yv and the V archive written
        return "hbm", 4.0 * P + 4.0 * (n + 1) + 5.0 * esz * n + esz * S * (8 * n + 2 * m)
    if name == "k_update":      # Y, x_{j-1}, x_{j-2} read and x_j written, vertex records and star rows
        return "hbm", esz * S * (8 * n + 4 * m) + esz * (2 * n + m)
    if name == "k_krylov_steps":  # all k steps in one launch, plus the last archive
        step = sum(kernel_model(x, H, K, S, k, esz)[1]
                   for x in ("k_edge_pass", "k_node_pass", "k_update"))
        return "hbm", k * step + 2.0 * n * S * esz * 2
    return "hbm", float("nan")


# ---------------------------------------------------------------- reference arm (oracle)

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import hef_oracle as O
    H, k, S = instance(args.workload, 0)
    # each step is the oracle on a window of the workload, sized so that the
    # whole run takes about 100 s (at most 3 s per step): a probe on a
    # 125 x 105 window gives the cost per pin
    Hp = window_subhypergraph(H, 0, min(H.nx, 125), 0, min(H.ny, 105)) if H.nx else H
    xp, xq = start_block(Hp.n, Hp.m, S, 0)
    t0 = time.perf_counter()
    O.hyperedge_resistance(Hp.n, Hp.eptr, Hp.pins, Hp.w, xp, xq, k)
    per_pin = (time.perf_counter() - t0) / max(Hp.P, 1)
    budget = min(3.0, 100.0 / max(args.steps + args.warmup, 1))
    frac = min(1.0, budget / (per_pin * H.P))
    rows = max(20, int(H.ny * frac)) if H.nx else 0
    Hs = window_subhypergraph(H, 0, H.nx, 0, min(H.ny, rows)) if H.nx else H
    x0c, x0b = start_block(Hs.n, Hs.m, S, 0)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.hyperedge_resistance(Hs.n, Hs.eptr, Hs.pins, Hs.w, x0c, x0b, k)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    v = Hs.P / t
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "pins/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample": f"{Hs.nx}x{Hs.ny} window",
                   "n": Hs.n, "m": Hs.m, "P": Hs.P, "k": k, "S": S, "K": 2 * k * S},
        "cpu_baseline": {"value": v, "unit": "pins/s", "cores": os.cpu_count(),
                         "kind": "oracle",
                         "sample": f"{Hs.nx}x{Hs.ny} window of the workload "
                                   f"(n={Hs.n}, m={Hs.m}, P={Hs.P}); numpy/scipy FP64, "
                                   "BLAS calls on all cores"},
        "e2e": {"value": v, "unit": "pins/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(name):
    """The oracle on the whole workload (one run, about 10 s on 16 cores)."""
    from oracle import hef_oracle as O
    H, k, S = instance(name, 0)
    x0c, x0b = start_block(H.n, H.m, S, 0)
    t0 = time.perf_counter()
    O.hyperedge_resistance(H.n, H.eptr, H.pins, H.w, x0c, x0b, k)
    t = time.perf_counter() - t0
    return {"value": H.P / t, "unit": "pins/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"the whole workload (n={H.n}, m={H.m}, P={H.P}), one run, "
                      f"{t:.1f} s; numpy/scipy FP64, BLAS calls on all cores"}


# ---------------------------------------------------------------- our arm

def score_errors(R, ref):
    big = ref >= 1e-3 * ref.max()
    rel = np.abs(R - ref) / np.maximum(ref, 1e-300)
    from scipy.stats import kendalltau
    return {"max_rel": float(rel[big].max()), "p99_rel": float(np.percentile(rel[ref > 0], 99)),
            "normwise": float(np.abs(R - ref).max() / ref.max()),
            "kendall_tau": float(kendalltau(R, ref).statistic)}


def precision_leg(hef, args, dev, rank, timed, max_ranks, world):
    """The precision form at its own scale: the 1200 x 1000 grid with 1.3M
    nets (2 + Geometric(0.5) pins, radius 3), k = 24, S = 8 (K = 384), FP32
    basis with tensor-core or FP32 Gram, FP64 Cholesky and Q_H; one CUDA
    graph per step.  Against it: the FP64 form on the same instance (one
    step), and the FP64 oracle on the induced 400 x 250 window (100k cells)
    scored by the same FP32 path."""
    import torch
    name = "grid1200x1000_m1300k"
    H, k, S = instance(name, rank)
    K = 2 * k * S
    x0c, x0b = start_block(H.n, H.m, S, 3 + rank)
    t = dict(eptr=torch.from_numpy(H.eptr).to(dev), pins=torch.from_numpy(H.pins).to(dev),
             w=torch.from_numpy(H.w).to(dev), x0c=torch.from_numpy(x0c).to(dev),
             x0b=torch.from_numpy(x0b).to(dev))
    pipe = hef.Pipeline(H.n, H.m, H.P, k, S, torch.float32, device=dev)
    pipe.run(t["eptr"], t["pins"], t["w"], t["x0c"], t["x0b"])
    torch.cuda.synchronize()
    pipe.check()
    hef.trace_read()
    hef.trace_kernels("k_")
    pipe.run(t["eptr"], t["pins"], t["w"], t["x0c"], t["x0b"])
    torch.cuda.synchronize()
    hef.trace_kernels(None)
    per_kernel = {k_: round(v[1], 3) for k_, v in
                  sorted(hef.trace_read().items(), key=lambda kv: -kv[1][1])[:8]}
    pipe.capture(t["eptr"], t["pins"], t["w"], t["x0c"], t["x0b"])
    ms, _, _, _ = timed(pipe.replay, args.steps, args.warmup)
    t32 = max_ranks(sum(ms) / len(ms))
    R32 = pipe.out["R"].cpu().numpy()
    rank32 = int(pipe.rank.item())
    del pipe
    p64 = hef.Pipeline(H.n, H.m, H.P, k, S, torch.float64, device=dev)
    step64 = lambda: p64.run(t["eptr"], t["pins"], t["w"], t["x0c"], t["x0b"])  # noqa
    ms64, _, _, _ = timed(step64, 1, 1)
    t64 = max_ranks(sum(ms64) / len(ms64))
    R64 = p64.out["R"].cpu().numpy()
    del p64
    out = {"workload": name, "n": H.n, "m": H.m, "P": H.P, "k": k, "S": S, "K": K,
           "dtype": "f32 basis, FP64 Cholesky and Q_H", "rank": rank32, "ms_per_step": t32,
           "pins_per_s": world * H.P / (t32 * 1e-3),
           "fp64_plain": {"ms_per_step": t64, "pins_per_s": world * H.P / (t64 * 1e-3)},
           "speedup_vs_fp64": t64 / t32, "error_vs_fp64_gpu": score_errors(R32, R64),
           "top_kernels_ms_one_step": per_kernel}
    # the BF16-storage form on the same instance (FP32 chains archived in
    # BF16, tensor-core CholQR2 on BF16 operands, FP32 spreads from BF16 loads)
    pb = hef.Pipeline(H.n, H.m, H.P, k, S, torch.bfloat16, device=dev)
    pb.run(t["eptr"], t["pins"], t["w"], t["x0c"], t["x0b"])
    torch.cuda.synchronize()
    pb.check()
    hef.trace_read()
    hef.trace_kernels("k_")
    pb.run(t["eptr"], t["pins"], t["w"], t["x0c"], t["x0b"])
    torch.cuda.synchronize()
    hef.trace_kernels(None)
    per_kernel_bf = {k_: round(v[1], 3) for k_, v in
                     sorted(hef.trace_read().items(), key=lambda kv: -kv[1][1])[:8]}
    pb.capture(t["eptr"], t["pins"], t["w"], t["x0c"], t["x0b"])
    msb, _, _, _ = timed(pb.replay, args.steps, args.warmup)
    tbf = max_ranks(sum(msb) / len(msb))
    Rbf = pb.out["R"].cpu().numpy()
    rankbf = int(pb.rank.item())
    del pb
    ebf = score_errors(Rbf, R64)
    out["bf16"] = {"dtype": "bf16 basis (FP32 chains, spreads and Gram accumulation; FP64 Cholesky "
                            "and Q_H)", "rank": rankbf, "ms_per_step": tbf,
                   "pins_per_s": world * H.P / (tbf * 1e-3), "speedup_vs_fp64": t64 / tbf,
                   "error_vs_fp64_gpu": ebf,
                   "meets_2e-3": bool(ebf["max_rel"] <= 2e-3 and ebf["p99_rel"] <= 2e-3),
                   "top_kernels_ms_one_step": per_kernel_bf}
    if rank == 0 and not args.no_precision_oracle:
        from oracle import hef_oracle as O
        Hs = window_subhypergraph(H, 0, 400, 0, 250)
        xs, xb = start_block(Hs.n, Hs.m, S, 3)
        tw = dict(eptr=torch.from_numpy(Hs.eptr).to(dev), pins=torch.from_numpy(Hs.pins).to(dev),
                  w=torch.from_numpy(Hs.w).to(dev), x0c=torch.from_numpy(xs).to(dev),
                  x0b=torch.from_numpy(xb).to(dev))
        win = {}
        for label, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
            o = hef.hyperedge_resistance(Hs.n, tw["eptr"], tw["pins"], tw["w"], tw["x0c"],
                                         tw["x0b"], k, dt)
            win[label] = o["R"].cpu().numpy()
        t0 = time.perf_counter()
        ref = O.hyperedge_resistance(Hs.n, Hs.eptr, Hs.pins, Hs.w, xs, xb, k)["R"]
        osec = time.perf_counter() - t0
        out["error_vs_oracle_window"] = dict(score_errors(win["f32"], ref), n=Hs.n, m=Hs.m,
                                             window="400x250", oracle_s=osec)
        eb = score_errors(win["bf16"], ref)
        out["bf16"]["error_vs_oracle_window"] = dict(
            eb, n=Hs.n, m=Hs.m, window="400x250",
            meets_2e3=bool(eb["max_rel"] <= 2e-3 and eb["p99_rel"] <= 2e-3))
    return out


def batched_leg(hef, args, dev, rank, timed, max_ranks, world):
    """The batched form: G netlists of uneven sizes (n log-uniform in
    5k..150k, m = 1.05 n, 2 + Geometric(0.5) pins on radius-3 neighbourhoods,
    unit weights; k = 20, S = 4), scored in one hef_resistance_batched call
    captured as a CUDA graph with the autotuned stream count and schedule,
    FP32.  Against it: the same batch in FP64 on one stream (the plain form,
    one netlist after another), and the error of FP32 against FP64."""
    import torch
    from netlists.synth import batch_sizes, grid_netlist
    k, S = 20, 4
    graphs = []
    P = 0
    for g, (nx, ny, m, seed) in enumerate(batch_sizes(args.batched_graphs, 4000 + 1000 * rank)):
        H = grid_netlist(nx, ny, m, seed)
        x0c, x0b = start_block(H.n, H.m, S, seed)
        graphs.append(dict(n=H.n, eptr=torch.from_numpy(H.eptr).to(dev),
                           pins=torch.from_numpy(H.pins).to(dev), w=torch.from_numpy(H.w).to(dev),
                           x0c=torch.from_numpy(x0c).to(dev), x0b=torch.from_numpy(x0b).to(dev)))
        P += H.P
    n_tot = sum(gr["n"] for gr in graphs)
    b32 = hef.Batch(graphs, k, S, torch.float32)
    b32.run()
    torch.cuda.synchronize()
    b32.check()
    # each Krylov form at 16 streams (graph replays), then the autotuner's pick
    forms = {}
    for form in (1, 0):
        hef.set_batch_krylov_form(form)
        bf = hef.Batch(graphs, k, S, torch.float32, nstreams=16)
        bf.run()
        bf.capture()
        msf, _, _, _ = timed(bf.replay, max(2, args.steps // 4), 1)
        forms["one_launch" if form else "per_step"] = round(statistics.median(msf), 3)
        del bf
    hef.set_batch_krylov_form(1)
    ns, _, tune_ms = b32.autotune()
    form = hef.batch_krylov_form()
    # launches and the top kernels of one eager run with the chosen settings
    hef.trace_read()
    hef.trace_kernels("k_")
    l0 = hef.launch_count()
    b32.run()
    torch.cuda.synchronize()
    launches = hef.launch_count() - l0
    hef.trace_kernels(None)
    top = {k_: round(v[1], 3) for k_, v in
           sorted(hef.trace_read().items(), key=lambda kv: -kv[1][1])[:8]}
    b32.capture()
    ms, _, _, _ = timed(b32.replay, args.steps, args.warmup)
    t32 = max_ranks(sum(ms) / len(ms))
    R32 = [o["R"].double().cpu().numpy() for o in b32.out]
    del b32
    # the FP64 form on the same schedule (streams and Krylov form)
    b64 = hef.Batch(graphs, k, S, torch.float64, nstreams=ns)
    b64.run()
    torch.cuda.synchronize()
    b64.capture()
    ms64, _, _, _ = timed(b64.replay, max(1, args.fp64_steps), 1)
    t64 = max_ranks(sum(ms64) / len(ms64))
    R64 = [o["R"].cpu().numpy() for o in b64.out]
    del b64
    a = np.concatenate(R32)
    r = np.concatenate(R64)
    big = r >= 1e-3 * r.max()
    rel = np.abs(a - r) / np.maximum(r, 1e-300)
    norm = max(float(np.abs(x - y).max() / y.max()) for x, y in zip(R32, R64))
    hef.set_batch_krylov_form(1)
    return {"graphs": len(graphs), "n_total": n_tot, "P_total": P, "k": k, "S": S,
            "dtype": "f32", "nstreams": ns,
            "krylov_form": "one cooperative launch for all netlists" if form else
                           "per-step launches per netlist",
            "ms_per_batch_by_form_16_streams": forms, "launches_per_batch": launches,
            "top_kernels_ms_eager_batch": top,
            "autotune_ms": tune_ms, "ms_per_batch": t32,
            "pins_per_s": world * P / (t32 * 1e-3),
            "fp64_same_schedule": {"ms_per_batch": t64, "pins_per_s": world * P / (t64 * 1e-3)},
            "speedup_vs_fp64": t64 / t32,
            "error_vs_fp64": {"max_rel": float(rel[big].max()),
                              "p99_rel": float(np.percentile(rel[r > 0], 99)),
                              "normwise_worst_graph": norm}}


def backward_leg(hef, args, dev, rank, timed, max_ranks, world):
    """FP32 forward (keeping the Krylov tape) and backward of
    L = sum over a seeded 10 % subset of w_e R_e, on the log-uniform-weight
    netlist; dL/dR = w_e on the subset.  Times forward and backward with CUDA
    events (L2 flushed before each step) and reports the Euler identity
    sum_e w_e dL/dw_e = -L of the score term as a live check."""
    import torch
    H, k, S = instance(args.backward_workload, rank)
    K = 2 * k * S
    x0c, x0b = start_block(H.n, H.m, S, 5 + rank)
    t = dict(eptr=torch.from_numpy(H.eptr).to(dev), pins=torch.from_numpy(H.pins).to(dev),
             w=torch.from_numpy(H.w).to(dev), x0c=torch.from_numpy(x0c).to(dev),
             x0b=torch.from_numpy(x0b).to(dev))
    sel = np.random.default_rng(5).random(H.m) < 0.1
    g = torch.from_numpy(np.where(sel, H.w, 0.0)).to(dev)
    state = {}

    def fwd():
        inc = hef.build_incidence(H.n, t["eptr"], t["pins"], t["w"])
        V, tape = hef.krylov_basis_tape(inc, t["x0c"], t["x0b"], k, torch.float32)
        Q, Rf, _ = hef.orthonormalize(V, K, want_R=True)
        sc = hef.edge_resistance(inc, Q, K)
        state.update(inc=inc, Q=Q, Rf=Rf, sc=sc, tape=tape)

    def bwd():
        s_ = state
        s_["grad"] = hef.edge_resistance_backward(s_["inc"], k, t["x0c"], t["x0b"], s_["Q"],
                                                  s_["Rf"], s_["sc"], g, tape=s_["tape"])

    def step():
        fwd()
        bwd()

    ms_f, _, _, _ = timed(fwd, args.steps, args.warmup)
    ms_s, _, _, _ = timed(step, args.steps, 1)
    fwd()
    torch.cuda.synchronize()
    hef.trace_read()
    hef.trace_kernels("k_bwd")
    bwd()
    torch.cuda.synchronize()
    hef.trace_kernels(None)
    top_bwd = {k_: round(v[1], 3) for k_, v in
               sorted(hef.trace_read().items(), key=lambda kv: -kv[1][1])[:8]}
    tf = max_ranks(sum(ms_f) / len(ms_f))
    ts = max_ranks(sum(ms_s) / len(ms_s))
    torch.cuda.synchronize()
    state["inc"].check()
    dw = state["grad"][0].cpu().numpy()
    R = state["sc"]["R"].cpu().numpy()
    gn = g.cpu().numpy()
    L = float(gn @ R)
    euler = abs(float(H.w @ dw) + L) / L
    tape_mb = state["tape"].numel() / 2**20
    return {"workload": args.backward_workload, "n": H.n, "m": H.m, "P": H.P, "k": k, "S": S,
            "dtype": "f32 basis, QR and chain adjoints; FP64 scoring adjoint", "loss": "sum over a seeded 10% subset of w_e R_e",
            "ms_forward": tf, "ms_forward_backward": ts, "ms_backward": ts - tf,
            "pins_per_s_forward_backward": world * H.P / (ts * 1e-3),
            "tape_mib": tape_mb, "euler_residual": euler, "top_backward_kernels_ms": top_bwd}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    import paper_2511_06600_gb300 as hef

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    H, k, S = instance(args.workload, rank)
    K = 2 * k * S
    x0c, x0b = start_block(H.n, H.m, S, rank)
    t_in = dict(eptr=torch.from_numpy(H.eptr).to(dev), pins=torch.from_numpy(H.pins).to(dev),
                w=torch.from_numpy(H.w).to(dev), x0c=torch.from_numpy(x0c).to(dev),
                x0b=torch.from_numpy(x0b).to(dev))
    dtype = torch.float32 if args.form == "f32" else torch.float64
    esz = 4 if args.form == "f32" else 8
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    max_ranks = lambda x: max_over_ranks(x, world, dev)  # noqa: E731
    P_all = sum_over_ranks(H.P, world, dev)  # pins scored by all ranks in one step

    def timed(fn, steps, warmup, trace=None):
        """Per-step CUDA-event times (ms) with an L2 flush before each step."""
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if trace:
            hef.trace_read()
            hef.trace_kernels(trace)
        barrier()
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        l0 = hef.launch_count()
        wall0 = time.perf_counter()
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record(st)
            fn()
            ev[i][1].record(st)
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - wall0
        launches = hef.launch_count() - l0
        tr = None
        if trace:
            hef.trace_kernels(None)
            tr = hef.trace_read()
        ms = [a.elapsed_time(b) for a, b in ev]
        return ms, launches, wall, tr

    # ---- main form: device-resident inputs
    pipe = hef.Pipeline(H.n, H.m, H.P, k, S, dtype, device=dev)
    eager = lambda: pipe.run(t_in["eptr"], t_in["pins"], t_in["w"], t_in["x0c"], t_in["x0b"])  # noqa
    step = eager
    # which kernel dominates: trace all library kernels over the warm-up steps
    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    pipe.check()
    hef.trace_read()
    hef.trace_kernels("k_")
    step()
    torch.cuda.synchronize()
    hef.trace_kernels(None)
    per_kernel = hef.trace_read()
    dominant = max(per_kernel.items(), key=lambda kv: kv[1][1])[0]
    per_kernel_launches = sum(v[0] for v in per_kernel.values())

    # the whole path as one CUDA graph (falls back to eager launches)
    graph = False
    if not args.no_graph:
        try:
            pipe.capture(t_in["eptr"], t_in["pins"], t_in["w"], t_in["x0c"], t_in["x0b"])
            step = pipe.replay
            graph = True
        except Exception as exc:  # noqa: BLE001
            print(f"graph capture failed, timing eager launches: {exc}", file=sys.stderr)
            step = eager
    clocks = Clocks(local)
    clocks.start()
    ms, launches, wall, _ = timed(step, args.steps, args.warmup)
    clk = clocks.stop()
    pipe.check()
    R32 = pipe.out["R"].double().cpu().numpy()
    t_step = max_ranks(sum(ms) / len(ms))
    value = P_all / (t_step * 1e-3)
    if graph:  # kernels inside a replayed graph are not counted by the library
        launches = int(round(per_kernel_launches)) * args.steps
    # dominant kernel's launch durations: eager steps with CUDA events around it
    _, _, _, tr = timed(eager, args.steps, 1, trace=dominant)

    # ---- roofline of the dominant kernel (live, same timed region)
    hbm_peak, peak_kind, sm_max = peaks()
    nl, tot = tr.get(dominant, (0, float("nan")))
    bound, units = kernel_model(dominant, H, K, S, k, esz)
    avg_s = (tot / max(nl, 1)) * 1e-3
    if bound == "hbm":
        achieved = units / avg_s / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None, "kernel": dominant,
                "peak_kind": peak_kind}
    else:
        alu_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # FP32 FMA lanes x 2 flops x max clock
        achieved = units / avg_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": None, "kernel": dominant,
                "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"}
    roof["launches"] = nl
    roof["avg_ms"] = tot / max(nl, 1)
    roof["traffic"] = recorded_traffic(dominant, args.workload, args.form)
    roof["algorithmic_bytes"] = units if bound == "hbm" else None

    # ---- latency of the small FP64 case (64 x 32 grid, 2,300 nets, k = 10,
    # S = 1), one CUDA graph per step, with the Krylov steps as one
    # persistent launch and as three launches per step
    small = {}
    Hs, ks, Ss = instance("grid64x32_m2300", rank)
    xs0, xs1 = start_block(Hs.n, Hs.m, Ss, rank)
    ts = dict(eptr=torch.from_numpy(Hs.eptr).to(dev), pins=torch.from_numpy(Hs.pins).to(dev),
              w=torch.from_numpy(Hs.w).to(dev), x0c=torch.from_numpy(xs0).to(dev),
              x0b=torch.from_numpy(xs1).to(dev))
    for label, mode in (("persistent", 1), ("per_step_launches", 0)):
        hef.set_krylov_persistent(mode)
        ps = hef.Pipeline(Hs.n, Hs.m, Hs.P, ks, Ss, torch.float64, device=dev)
        ps.run(ts["eptr"], ts["pins"], ts["w"], ts["x0c"], ts["x0b"])
        ps.capture(ts["eptr"], ts["pins"], ts["w"], ts["x0c"], ts["x0b"])
        ms_s, _, _, _ = timed(ps.replay, args.steps, args.warmup)
        ps.check()
        small[label + "_ms"] = max_ranks(statistics.median(ms_s))
        del ps
    hef.set_krylov_persistent(1)
    small.update(workload="grid64x32_m2300", dtype="f64", n=Hs.n, m=Hs.m, P=Hs.P, k=ks, S=Ss)

    # ---- plain FP64 form (speedup reference) and its agreement with the FP32 form
    pipe64 = hef.Pipeline(H.n, H.m, H.P, k, S, torch.float64, device=dev)
    step64 = lambda: pipe64.run(t_in["eptr"], t_in["pins"], t_in["w"], t_in["x0c"], t_in["x0b"])  # noqa
    ms64, _, _, _ = timed(step64, args.fp64_steps, 1)
    pipe64.check()
    R64 = pipe64.out["R"].cpu().numpy()
    t64 = max_ranks(sum(ms64) / len(ms64))
    big = R64 >= 1e-3 * R64.max()
    rel = np.abs(R32 - R64) / np.maximum(R64, 1e-300)
    err = {"max_rel": float(rel[big].max()), "p99_rel": float(np.percentile(rel[R64 > 0], 99)),
           "normwise": float(np.abs(R32 - R64).max() / R64.max())}
    del pipe64

    # ---- end to end through the C ABI's host-array call (hef_resistance_host):
    # pinned host inputs in, the whole path, the scores back in host memory
    e2e = None
    if not args.no_e2e:
        host = {key: t.cpu().pin_memory() for key, t in t_in.items()}
        R_host = torch.empty(H.m, dtype=torch.float64).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        d2h = R_host.numel() * R_host.element_size()
        ws_host = hef.resistance_host_workspace(H.n, H.m, H.P, k, S, dtype, device=dev)

        def e2e_step():
            hef.resistance_host(H.n, host["eptr"], host["pins"], host["w"], host["x0c"],
                                host["x0b"], k, dtype, R_out=R_host, workspace=ws_host)

        ms_e, _, _, _ = timed(e2e_step, args.steps, 1)
        te = max_ranks(sum(ms_e) / len(ms_e))
        assert np.allclose(R_host.numpy(), R32, rtol=1e-4, atol=0), "host-array call disagrees"
        e2e = {"value": P_all / (te * 1e-3), "unit": "pins/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": te,
               "call": "hef_resistance_host (host arrays in, R out, one synchronisation)"}

    # ---- differentiation form: forward + backward of a score-based loss
    bwd = None
    if not args.no_backward:
        bwd = backward_leg(hef, args, dev, rank, timed, max_ranks, world)

    # ---- precision form at its own scale (1.2M cells, K = 384)
    precision = None
    if not args.no_precision:
        precision = precision_leg(hef, args, dev, rank, timed, max_ranks, world)

    # ---- batched form: many uneven netlists in one captured call
    batched = None
    if not args.no_batched:
        batched = batched_leg(hef, args, dev, rank, timed, max_ranks, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "pins/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.form, "data": "synthetic",
            "config": {"workload": args.workload, "n": H.n, "m": H.m, "P": H.P, "k": k, "S": S,
                       "K": K, "form": args.form + " storage/accumulation, FP64 Cholesky and Q_H",
                       "l2": f"flushed before every step ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "parallelism": f"{world} independent netlists (one per GPU)"},
            "scores_per_s": world * H.m / (t_step * 1e-3),
            "fp64_plain": {"value": P_all / (t64 * 1e-3), "unit": "pins/s",
                           "ms_per_step": t64},
            "speedup_vs_fp64": t64 / t_step,
            "small_fp64_latency": small,
            "error_vs_fp64": err,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "backward": bwd,
            "batched": batched,
            "precision": precision,
            "gpu_launches": launches,
            "cuda_graph": graph,
            "launches_per_step": launches / max(args.steps, 1),
            "per_kernel_ms_one_step": {k_: round(v[1], 4) for k_, v in
                                       sorted(per_kernel.items(), key=lambda kv: -kv[1][1])},
            "clocks": clk,
            "wall_s_timed_region": wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
