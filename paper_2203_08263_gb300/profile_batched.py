"""Run the batched ensemble once, for timing and profiling.

    python -m paper_2203_08263_gb300.profile_batched [--steps 100] [--tune] [--form pair_symmetric]

Input: 512 uniform-cube systems with N log-uniform in [64, 8192] (seed 3),
eps = 0.01, dt = 1e-3. Prints the CUDA-event time of one nb_run_batched call
and the rate in body-pair interactions per second (sum of N_s^2 per step).
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--nsys", type=int, default=512)
    ap.add_argument("--tune", action="store_true", help="autotune the batched shape first")
    ap.add_argument("--form", default=None, choices=["one_sided", "pair_symmetric"],
                    help="pin the batched form (default: chosen for the sizes)")
    a = ap.parse_args()

    import torch

    from paper_2203_08263_gb300 import build, ics
    from paper_2203_08263_gb300.nbody import Context

    build.build()
    dev = torch.device("cuda:0")
    off, x, v, m = ics.ensemble(a.nsys, 3)
    ctx = Context(1.0, 0.01, 1e-3)
    offt = torch.tensor(off, dtype=torch.int64)
    if a.tune:
        ctx.autotune_batched(offt)
    if a.form:
        ctx.set_batched_form(offt, a.form)
    xt, vt, mt = (torch.tensor(t, dtype=torch.float32, device=dev) for t in (x, v, m))
    ctx.run_batched(offt, xt.clone(), vt.clone(), mt, 1)  # plan and capture
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx.run_batched(offt, xt, vt, mt, a.steps)
    e1.record()
    torch.cuda.synchronize()
    ctx.sync()
    t = e0.elapsed_time(e1) / 1e3
    inter = float((np.diff(off).astype(np.float64) ** 2).sum()) * a.steps
    print(json.dumps({"systems": a.nsys, "bodies": int(off[-1]), "steps": a.steps, "s": t,
                      "interactions_per_s": inter / t, "shape": ctx.get_batched_config(offt)}))


if __name__ == "__main__":
    main()
