#!/usr/bin/env python
"""Benchmark of the all-pairs N-body step on GB300 (one JSON line on stdout).

Workload (default): single large system, N = 262144 Plummer sphere (seed 1),
G = 1, eps = 0.05, dt = 1e-3, FP32. One bench step = one step of the paper's
update through the library (pack + force sum + half kick + drift). Metric:
body-pair interactions per second, N^2 per step (self pairs counted, as the
paper's 20 N^2 I / t GFLOPS convention does), and the fraction of the FP32
FMA peak at 20 flops per interaction.

--impl reference times the FP64 CPU oracle on the host cores instead, each
step on a bounded sample of the same workload (a subset of i-bodies against
all N j-bodies).

Under torchrun each rank runs an independent replica on its own GPU (the
single-system path has no exchange on one GPU); value sums the ranks'
interactions over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Body-pair interactions/s and % of FP32 peak; adjoint-to-forward time ratio"
UNIT = "interactions/s"
FLOPS_PER_INTERACTION = 20  # the paper's convention (Section 4.1)


def workload(n: int) -> str:
    return (f"single system N={n} Plummer (seed 1), G=1, eps=0.05, dt=1e-3; "
            "one bench step = one paper update (force sum + half kick + drift)")


L2_NOTE = ("GPU arm: L2 flushed between timed steps (256 MiB write outside the timed events); "
           "CPU reference arm: each step a fresh i-sample against the whole j-array")


def bench_config(n: int, world: int) -> dict:
    """The workload keys, identical in both arms (launch details go under
    "launch" in the GPU arm's line)."""
    return {"workload": workload(n), "n": n, "l2": L2_NOTE,
            "parallelism": "single GPU" if world == 1 else f"{world} independent replicas, one per GPU"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=262144)
    ap.add_argument("--no-extras", action="store_true", help="skip the C3/C4/C5 side measurements")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def cpu_baseline(n_all, x, m, G, eps, seconds=10.0):
    """The FP64 oracle as it stands, on every host core, over i-subsets of the
    same system until `seconds` of work are done."""
    import numpy as np

    import oracle

    chunk = 512
    done_i = 0
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < seconds:
        idx = np.arange(k * chunk, (k + 1) * chunk) % n_all
        oracle.accel(x, m, G, eps, idx)
        done_i += chunk
        k += 1
    dt = time.perf_counter() - t0
    return {"value": done_i * n_all / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"FP64 force sum of {done_i} i-bodies (chunks of {chunk}) against all {n_all} bodies "
                      f"of the same system, {dt:.1f} s"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2203_08263_gb300 import ics

    oracle.build()
    n, G, eps = args.n, 1.0, 0.05
    s = ics.plummer(n, seed=1)
    sample = 2048
    times = []
    for k in range(args.warmup + args.steps):
        idx = (np.arange(sample) * 127 + k * sample) % n
        t0 = time.perf_counter()
        oracle.accel(s.x, s.m, G, eps, idx)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = sample * n * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(n, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"each step: the FP64 oracle's force sum for {sample} i-bodies "
                                   f"against all {n} j-bodies (a bounded sample of one step)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# DRAM bytes per launch of the step kernel (force sum + kick/drift epilogue)
# at N = 262144, by launch shape (threads, bodies/thread, j-split, j-tile):
# ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch each, on this
# GPU type. Most of it is split partials evicted from L2; the O(N) state is
# 21 MB. Reported only when the bench runs one of these shapes.
# The pair-symmetric kernel (threads, 8, 1, block) writes nb x 3 x npad floats
# of block-pair partials (0.8 GB at N = 262144); its entry is a one-pass
# capture at N = 262144 with L2 contents carried between kernels
# (--cache-control none), the mean of two launches.
STEP_TRAFFIC_BYTES = {
    (128, 8, 1, 1024): 5.53e6 + 773.9e6,
    (128, 8, 19, 128): 11.85e6 + 34.15e6,
    (128, 8, 19, 64): 11.07e6 + 34.31e6,
    (128, 4, 16, 256): 11.16e6 + 21.29e6,
    (128, 8, 19, 256): 11.77e6 + 34.34e6,
    (128, 8, 26, 256): 12.73e6 + 63.50e6,
    (256, 2, 16, 256): 10.96e6 + 21.27e6,
}
# The pair-symmetric kernel by tiles (above 512 MiB of one-launch partials),
# by (shape, launches per step): DRAM bytes per step, summed over the step's
# tile launches of the pair kernel, the final fold and the pack (one-pass
# capture at N = 262144 as above).
STEP_TRAFFIC_TILED = {
    ((128, 8, 1, 1024), 68): 0.02e6 + 19.57e6,  # 66 tiles of 24 x 24 block pairs
}


FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2070e6 / 1e12  # unit counts x maximum SM clock

# FP32 lane operations per ordered interaction, by force form: the one-sided
# kernel spends 3 subtractions, 3 multiply-adds for s, 3 multiplies for
# m s^-3/2 and 3 multiply-adds into a (12); the pair-symmetric kernel spends
# 16 per unordered pair (d, s and s^-3/2 shared), 8 per ordered interaction.
OPS_PER_INTERACTION = {"f32x2": 12, "scalar": 12, "pair_symmetric": 8}
KERNEL_NAME = {"f32x2": "force_kernel<AccelF32x2> (+ its 1-launch pack, <0.1% of the step)",
               "scalar": "force_kernel<AccelScalar> (+ its 1-launch pack)",
               "pair_symmetric": "sym_force_kernel (+ sym_finish_kernel, the fixed-order sum of the "
                                 "block-pair partials with the kick/drift epilogue, and the pack: "
                                 "timed together, so the kernel's own rate is slightly higher)",
               "pair_symmetric_tiled": "sym_force_kernel by tiles of block pairs (one launch per tile, "
                                       "each folding the previous tile's partials into running sums) "
                                       "+ sym_tile_final_kernel (the last fold with the kick/drift "
                                       "epilogue) + the pack: timed together"}


def fp32_peak_tflops(props, sm_max_mhz):
    # 128 FP32 lanes per SM, 2 flops per FMA, at the maximum SM clock
    return props.multi_processor_count * 128 * 2 * sm_max_mhz * 1e6 / 1e12


def use_shipped_tuning_table(torch, device: int) -> str:
    """Point the library at the tuner's table for this GPU type, when the
    package ships one (written by paper_2203_08263_gb300.tune_table on this
    GPU type): launch shapes then come from the tuner and are reproducible.
    A private copy is used so that no run rewrites the shipped file."""
    import shutil

    from paper_2203_08263_gb300.tune_table import table_path

    if os.environ.get("NB_AUTOTUNE_CACHE"):
        return "NB_AUTOTUNE_CACHE"
    src = table_path(torch.cuda.get_device_name(device))
    if not os.path.exists(src):
        return "none"
    fd, tmp = tempfile.mkstemp(suffix=".json")
    os.close(fd)
    shutil.copyfile(src, tmp)
    os.environ["NB_AUTOTUNE_CACHE"] = tmp
    return "tuner table shipped for this GPU type"


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2203_08263_gb300 import build as nbuild
    from paper_2203_08263_gb300 import ics
    from paper_2203_08263_gb300.nbody import Context

    nbuild.build()
    shape_source = use_shipped_tuning_table(torch, local)
    n, G, eps, dt = args.n, 1.0, 0.05, 1e-3
    s = ics.plummer(n, seed=1)
    ctx = Context(G, eps, dt, device=local)
    if not ctx.get_config(n)["tuned"]:
        ctx.autotune(n)
        shape_source = "tuned in this run"
    cfg = ctx.get_config(n)
    x = torch.tensor(s.x, dtype=torch.float32, device=dev)
    v = torch.tensor(s.v, dtype=torch.float32, device=dev)
    m = torch.tensor(s.m, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        ctx.run(x, v, m, 1)
    torch.cuda.synchronize(dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    clocks = Clocks(local)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = ctx.launch_count
    barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    for k in range(args.steps):
        flush.fill_(float(k))  # L2 flush between steps, outside the timed events
        evs[k][0].record(stream)
        ctx.run(x, v, m, 1)
        evs[k][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    launches = ctx.launch_count - l0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    tot_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([tot_ms], dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        tot_ms = float(t.item())
    inter = float(n) * n
    value = world * inter * args.steps / (tot_ms / 1e3)
    ms_step = tot_ms / args.steps

    props = torch.cuda.get_device_properties(dev)
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak_20 = fp32_peak_tflops(props, sm_max)
    form = cfg.get("form", "f32x2")
    ops = OPS_PER_INTERACTION.get(form, 12)
    # the FP32 pipe's roofline: lane operations the form executes per second
    # against 128 lanes per SM per clock
    lane_peak = props.multi_processor_count * 128 * sm_max * 1e6 / 1e12
    achieved = ops * inter / (ms_step / 1e3) / 1e12
    shape_key = (cfg["threads"], cfg["bodies_per_thread"], cfg["split"], cfg["jtile"])
    per_step = round(launches / args.steps)
    tiled = form == "pair_symmetric" and per_step > 3  # pack, the tiles, the final fold
    if tiled:
        traffic = STEP_TRAFFIC_TILED.get((shape_key, per_step)) if n == 262144 else None
        traffic_unit = (f"bytes per step ({per_step - 2} tile launches of the pair kernel, "
                        "the final fold and the pack)")
    else:
        traffic = STEP_TRAFFIC_BYTES.get(shape_key) if n == 262144 else None
        traffic_unit = "bytes per launch"
    roofline = {"bound": "alu", "achieved": achieved, "peak": lane_peak, "unit": "T FP32 lane-ops/s",
                "frac": achieved / lane_peak, "traffic": traffic, "traffic_unit": traffic_unit,
                "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x {sm_max:.0f} MHz "
                              f"(max SM clock); {ops} lane operations per interaction in the {form} form",
                "kernel": KERNEL_NAME.get(form + ("_tiled" if tiled else ""), form),
                "pct_fp32_peak_20flop": 100.0 * FLOPS_PER_INTERACTION * inter / (ms_step / 1e3) / 1e12 / peak_20,
                "pct_basis": f"20 flops per interaction (Section 4.1) over {peak_20:.2f} TFLOP/s "
                             "(2 flops per FMA lane); above the one-sided form's 83.3 % ceiling when "
                             "each pair term feeds two bodies"}

    # end to end through the public C-ABI with host buffers: the call copies
    # the state in, runs the step, copies it back and returns
    xh = torch.tensor(s.x, dtype=torch.float32).pin_memory().numpy()
    vh = torch.tensor(s.v, dtype=torch.float32).pin_memory().numpy()
    mh = torch.tensor(s.m, dtype=torch.float32).pin_memory().numpy()
    ctx.run(xh, vh, mh, 1)
    ke = max(3, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        ctx.run(xh, vh, mh, 1)
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * inter * ke / e2e_s, "unit": UNIT, "h2d_bytes_per_step": n * 4 * 7,
           "d2h_bytes_per_step": n * 4 * 6, "steps": ke}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(n, world),
        "launch": {"shape": cfg, "shape_source": shape_source},
        "roofline": roofline,
        "interactions_per_s_per_gpu": inter * args.steps / (tot_ms / 1e3),
        "gflops_20": FLOPS_PER_INTERACTION * value / 1e9,
        "clocks": clk, "gpu_launches": launches, "e2e": e2e,
    }

    c3_sample = c5_check = None
    if rank == 0 and world == 1 and not args.no_extras:
        line["extras"] = extras(ctx, torch, dev, np)
        c3_sample = line["extras"].pop("_c3_sample")
        c5_check = line["extras"].pop("_c5_check")
    if rank == 0 and world == 1 and not args.no_cpu:
        # the CPU-baseline leg: every oracle call of this arm
        line["cpu_baseline"] = cpu_baseline(n, s.x, s.m, G, eps)
        if "extras" in line:
            rows = oracle_rows(c3_sample, c5_check)
            line["extras"]["cpu_oracle_rows"] = rows
            line["extras"]["c3_precision_form"]["accel_rel_l2_vs_fp64_oracle_256_subset"] = \
                rows["c3_accuracy_sample"]["gpu_accel_rel_l2"]
            line["extras"]["c5_adjoint"]["gradient_rel_l2_vs_fp64_oracle_n64_T20"] = \
                rows["c5_gradient_check"]["gpu_gradient_rel_l2"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def _timed(torch, dev, fn, reps=1):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize(dev)
    return a.elapsed_time(b) / 1e3


def _adjoint_ratio(c, s, xs, f, T, k, torch, dev):
    """Wall time of T forward steps with a checkpoint every k (nb_run) and of
    the reverse sweep with its recompute (nb_adjoint) for the loss
    sum |x_T - x*|^2, on context c in state dtype f."""
    n = s.n
    x0, v0, m = (torch.tensor(a_, dtype=f, device=dev) for a_ in (s.x, s.v, s.m))
    ck = torch.empty((T // k + 1, n, 6), dtype=f, device=dev)
    x, v = x0.clone(), v0.clone()
    c.run(x, v, m, T, ckpt=ck, ckpt_every=k)
    xbT = 2 * (x - torch.tensor(xs, dtype=f, device=dev))
    vbT = torch.zeros_like(xbT)
    c.adjoint(m, T, ck, k, xbT, vbT)

    def fwd():
        x.copy_(x0)
        v.copy_(v0)
        c.run(x, v, m, T, ckpt=ck, ckpt_every=k)

    tf = _timed(torch, dev, fwd)
    tb = _timed(torch, dev, lambda: c.adjoint(m, T, ck, k, xbT, vbT))
    return {"n": n, "T": T, "k": k, "forward_s": tf, "backward_s": tb, "ratio": tb / tf,
            "forward_interactions_per_s": float(n) * n * T / tf,
            "forward_shape": c.get_config(n, 0), "vjp_shape": c.get_config(n, 1)}


def extras(ctx0, torch, dev, np):
    """Side measurements of the other rows: the precision form (C3), the
    batched ensemble (C4) and the adjoint-to-forward ratio (C5). The GPU
    forces on the C3 accuracy sample are returned under "_c3_sample" for the
    CPU-baseline leg, which holds every oracle call."""
    from paper_2203_08263_gb300 import ics
    from paper_2203_08263_gb300.nbody import Context

    out = {}
    # C1: plain method, small: N = 1024 cube (seed 0), 10 steps through nb_run
    # (the path the shipped tuning table picks: graph, one cluster or grid)
    s = ics.cube(1024, seed=0)
    c = Context(1.0, 0.01, 1e-3, device=dev.index)
    x, v, m = (torch.tensor(a, dtype=torch.float32, device=dev) for a in (s.x, s.v, s.m))
    c.run(x, v, m, 10)  # the timed call once (a graph path would capture its graph here)
    t = min(_timed(torch, dev, lambda: c.run(x, v, m, 10)) for _ in range(5))
    out["c1_small"] = {"n": 1024, "steps": 10, "s": t, "us_per_step": t / 10 * 1e6,
                       "interactions_per_s": 1024.0 * 1024 * 10 / t, "run_path": c.get_run_path(1024),
                       "graph_path_shape": c.get_config(1024)}
    c.close()
    # C3: precision form, N = 2^20 Plummer (seed 2), FP64 state, 10 steps
    n = 1 << 20
    s = ics.plummer(n, seed=2)
    c = Context(1.0, 0.05, 5e-4, precision="comp", device=dev.index)
    f = torch.float64
    x, v, m = (torch.tensor(a, dtype=f, device=dev) for a in (s.x, s.v, s.m))
    a = c.accel(x, m)
    idx = ics.subset_indices(n, 256, 2 + 1000)
    out["_c3_sample"] = (s.x, s.m, idx, a.cpu().numpy()[idx])
    x0, v0 = x.clone(), v.clone()
    c.run(x, v, m, 10)  # the timed call once: its step graph is captured here
    x.copy_(x0)
    v.copy_(v0)
    del x0, v0
    t = _timed(torch, dev, lambda: c.run(x, v, m, 10))
    out["c3_precision_form"] = {"n": n, "steps": 10, "interactions_per_s": 10 * float(n) * n / t, "s": t,
                                "shape": c.get_config(n)}
    # diagnostics on the C3 state: P, KE, softened potential (O(N^2)), H'
    t0 = time.perf_counter()
    e = c.energy(x, v, m)
    te = time.perf_counter() - t0
    out["c3_diagnostics"] = {"n": n, "s": te, "pairs_per_s": float(n) * n / te, "KE": e["KE"],
                             "Phi": e["Phi"], "H": e["H"], "P": [float(p_) for p_ in e["P"]]}
    c.close()
    del x, v, m, a
    # C4: batched ensemble, 512 systems, 100 steps, one persistent launch
    off, bx, bv, bm = ics.ensemble(512, 3)
    c = Context(1.0, 0.01, 1e-3, device=dev.index)
    xb, vb, mb = (torch.tensor(a_, dtype=torch.float32, device=dev) for a_ in (bx, bv, bm))
    offt = torch.tensor(off, dtype=torch.int64)
    c.autotune_batched(offt)  # threads, bodies per thread and j-tile from the project's tuner
    xb0, vb0 = xb.clone(), vb.clone()
    c.run_batched(offt, xb, vb, mb, 100)  # the timed call once: plan and capture
    xb.copy_(xb0)
    vb.copy_(vb0)
    t = _timed(torch, dev, lambda: c.run_batched(offt, xb, vb, mb, 100))
    sizes = np.diff(off).astype(np.float64)
    out["c4_batched"] = {"systems": 512, "bodies": int(off[-1]), "steps": 100,
                         "interactions_per_s": float((sizes ** 2).sum()) * 100 / t, "s": t,
                         "shape": c.get_batched_config(offt)}
    c.close()
    # C5: adjoint, N = 16384 cube (seed 4), T = 200, checkpoint every 20
    n, T, k = 16384, 200, 20
    s = ics.cube(n, seed=4, masses="equal")
    xs = ics.targets(n, seed=4)
    c = Context(1.0, 0.01, 1e-3, device=dev.index)
    for mode in (0, 1):  # forward and VJP shapes from the tuner
        if not c.get_config(n, mode)["tuned"]:
            c.autotune(n, mode)
    out["c5_adjoint"] = _adjoint_ratio(c, s, xs, torch.float32, T, k, torch, dev)
    c.close()
    # the same adjoint in the precision form (FP64 state and gradients,
    # compensated FP32 forces and VJP)
    c = Context(1.0, 0.01, 1e-3, precision="comp", device=dev.index)
    out["c5_adjoint_precision_form"] = _adjoint_ratio(c, s, xs, torch.float64, T, k, torch, dev)
    c.close()
    # gradients at the check size (N = 64, T = 20, k = 20) in both forms, for
    # the CPU-baseline leg to compare with the FP64 oracle's
    n, T, k = 64, 20, 20
    s = ics.cube(n, seed=4, masses="equal")
    xs = ics.targets(n, seed=4)
    grads = {}
    for prec, f in (("fp32", torch.float32), ("comp", torch.float64)):
        c = Context(1.0, 0.01, 1e-3, precision=prec, device=dev.index)
        x, v, m = (torch.tensor(a_, dtype=f, device=dev) for a_ in (s.x, s.v, s.m))
        ck = torch.empty((T // k + 1, n, 6), dtype=f, device=dev)
        c.run(x, v, m, T, ckpt=ck, ckpt_every=k)
        xbT = 2 * (x - torch.tensor(xs, dtype=f, device=dev))
        grads[prec] = [g.double().cpu().numpy() for g in c.adjoint(m, T, ck, k, xbT, torch.zeros_like(xbT))]
        c.close()
    out["_c5_check"] = (s, xs, grads)
    out["fp32_peak_fraction"] = {
        k: FLOPS_PER_INTERACTION * out[k]["interactions_per_s"] / 1e12 / FP32_PEAK_TFLOPS
        for k in ("c1_small", "c3_precision_form", "c4_batched")}
    return out


def oracle_rows(c3_sample=None, c5_check=None):
    """The FP64 oracle, as it stands, on bounded samples of the other rows
    (host cores of this machine), for comparison with the GPU rates above; with
    the GPU's C3 forces on the accuracy sample, their error against it."""
    import numpy as np

    import oracle
    from paper_2203_08263_gb300 import ics

    rows = {}
    if c3_sample is not None:
        x, m, idx, gpu = c3_sample
        t0 = time.perf_counter()
        ref = oracle.accel(x, m, 1.0, 0.05, idx)
        dt = time.perf_counter() - t0
        rows["c3_accuracy_sample"] = {
            "gpu_accel_rel_l2": float(np.linalg.norm(gpu - ref) / np.linalg.norm(ref)),
            "interactions_per_s": float(len(idx)) * len(x) / dt,
            "sample": f"{len(idx)} i x {len(x)} j (the bench's C3 accuracy subset)"}
    s = ics.plummer(1 << 20, seed=2)
    idx = ics.subset_indices(1 << 20, 512, 5)
    t0 = time.perf_counter()
    oracle.accel(s.x, s.m, 1.0, 0.05, idx)
    dt = time.perf_counter() - t0
    rows["c3_accel"] = {"interactions_per_s": 512.0 * (1 << 20) / dt, "sample": "512 i x 2^20 j"}
    off, x, v, m = ics.ensemble(512, 3)
    pick = np.argsort(np.diff(off))[-4:]
    t0 = time.perf_counter()
    inter = 0.0
    for sys_ in pick:
        a, b = off[sys_], off[sys_ + 1]
        oracle.run(x[a:b], v[a:b], m[a:b], 1.0, 0.01, 1e-3, 2)
        inter += 2.0 * (b - a) ** 2
    dt = time.perf_counter() - t0
    rows["c4_systems"] = {"interactions_per_s": inter / dt, "sample": "2 steps of the 4 largest systems"}
    n, T = 512, 20
    s = ics.cube(n, seed=4, masses="equal")
    t0 = time.perf_counter()
    oracle.adjoint(s.x, s.v, s.m, 1.0, 0.01, 1e-3, T, np.ones((n, 3)), np.zeros((n, 3)))
    dt = time.perf_counter() - t0
    rows["c5_adjoint"] = {"s": dt, "forward_interactions_per_s": float(n) * n * T / dt,
                          "sample": f"full adjoint (forward + reverse, explicit Jacobian blocks), N={n}, T={T}"}
    if c5_check is not None:
        s, xs, grads = c5_check
        t0 = time.perf_counter()
        xT, _ = oracle.run(s.x, s.v, s.m, 1.0, 0.01, 1e-3, 20)
        ref = oracle.adjoint(s.x, s.v, s.m, 1.0, 0.01, 1e-3, 20, 2 * (xT - xs), np.zeros((s.n, 3)))
        dt = time.perf_counter() - t0
        rows["c5_gradient_check"] = {
            "gpu_gradient_rel_l2": {
                prec: {name: float(np.linalg.norm(g - r) / np.linalg.norm(r))
                       for name, g, r in zip(("xbar0", "vbar0", "mbar"), grads[prec], ref)}
                for prec in grads},
            "s": dt, "sample": "N=64 cube (seed 4), T=20, checkpoint every 20: the FP64 oracle's run and "
                               "adjoint against the GPU gradients of both forms"}
    rows["cores"] = oracle.num_threads()
    return rows


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
