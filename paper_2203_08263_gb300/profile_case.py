"""Run one pair-sum kernel on a fixed launch shape, for timing and profiling.

    python -m paper_2203_08263_gb300.profile_case --n 65536 --shape 128,4,16,256 --pol fp32
    python -m paper_2203_08263_gb300.profile_case --n 1024 --pol step --steps 100 --path 2
    python -m paper_2203_08263_gb300.profile_case --n 262144 --pol step --steps 3 --form 1024
    python -m paper_2203_08263_gb300.profile_case --n 65536 --pol vjp --vjp-form 512
    python -m paper_2203_08263_gb300.profile_case --n 16384 --pol adjoint --steps 200
    python -m paper_2203_08263_gb300.profile_case --peaks

Input: Plummer sphere (seed 1), eps = 0.05. Prints the CUDA-event time per
call and the rate at 20 flops per interaction (--pol adjoint: one nb_adjoint
over a trajectory of --steps steps checkpointed every --ckpt-every, after
that trajectory is run). --form / --vjp-form pin the force form (one-sided or
a pair-symmetric block size); --tile sets the pair-symmetric launches (one
launch, or tiles of w x w block pairs). --peaks runs the FFMA, f32x2-FMA and MUFU
micro-benchmarks instead.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=65536)
    ap.add_argument("--shape", default="0,0,0,0", help="threads,bodies_per_thread,split,jtile (0 = auto)")
    ap.add_argument("--pol", default="fp32",
                    choices=["fp32", "comp", "vjp", "vjp-comp", "energy", "step", "step-comp", "adjoint"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--steps", type=int, default=1,
                    help="paper steps per call for --pol step / step-comp; T for --pol adjoint")
    ap.add_argument("--ckpt-every", type=int, default=20, help="checkpoint interval for --pol adjoint")
    ap.add_argument("--path", type=int, default=0,
                    help="nb_run path for --pol step / step-comp: 0 chosen per size, 1 graph, 2 one cluster")
    ap.add_argument("--form", type=int, default=0,
                    help="FP32 force form: 0 chosen per size, 1 one-sided, 512/1024 pair-symmetric blocks")
    ap.add_argument("--vjp-form", type=int, default=0,
                    help="FP32 VJP form: 0 chosen per size, 1 one-sided, 256/512 pair-symmetric blocks")
    ap.add_argument("--tile", type=int, default=0,
                    help="pair-symmetric launches: 0 chosen per size, -1 one launch, w tiles of w blocks")
    ap.add_argument("--peaks", action="store_true")
    a = ap.parse_args()

    import torch

    from paper_2203_08263_gb300 import build, ics
    from paper_2203_08263_gb300.nbody import (MODE_ADJOINT, MODE_FORWARD, MODE_POTENTIAL, NB_DBG_FORM,
                                              NB_DBG_RUN_PATH, NB_DBG_SYM_TILE, NB_DBG_VJP_FORM, Context)

    build.build()
    if a.peaks:
        ctx = Context(1.0, 0.05, 1e-3)
        runs = [ctx.measure_peaks() for _ in range(3)]
        print(json.dumps({"runs": runs, "best": {k: max(r[k] for r in runs) for k in runs[0]}}))
        return
    shape = tuple(int(v) for v in a.shape.split(","))
    prec = "comp" if a.pol in ("comp", "vjp-comp", "step-comp") else "fp32"
    f = torch.float64 if prec == "comp" else torch.float32
    dev = torch.device("cuda:0")
    s = ics.plummer(a.n, seed=1)
    ctx = Context(1.0, 0.05, 1e-3, precision=prec, tile_override=shape)
    ctx.debug_set(NB_DBG_RUN_PATH, a.path)
    ctx.debug_set(NB_DBG_FORM, a.form)
    ctx.debug_set(NB_DBG_VJP_FORM, a.vjp_form)
    ctx.debug_set(NB_DBG_SYM_TILE, a.tile)
    x, v, m = (torch.tensor(t, dtype=f, device=dev) for t in (s.x, s.v, s.m))
    ab = torch.tensor(np.random.default_rng(0).normal(size=(a.n, 3)), dtype=f, device=dev)
    mode = {"fp32": MODE_FORWARD, "comp": MODE_FORWARD, "vjp": MODE_ADJOINT, "vjp-comp": MODE_ADJOINT,
            "energy": MODE_POTENTIAL, "step": MODE_FORWARD, "step-comp": MODE_FORWARD,
            "adjoint": MODE_ADJOINT}[a.pol]
    if a.pol == "adjoint":  # a trajectory with checkpoints, then its reverse sweep (timed)
        k = a.ckpt_every
        ck = torch.empty((a.steps // k + 1, a.n, 6), dtype=f, device=dev)
        ctx.run(x, v, m, a.steps, ckpt=ck, ckpt_every=k)
        xb = torch.tensor(np.random.default_rng(1).normal(size=(a.n, 3)), dtype=f, device=dev)
        vb = torch.zeros_like(xb)

    def call():
        if a.pol in ("fp32", "comp"):
            ctx.accel(x, m)
        elif a.pol in ("vjp", "vjp-comp"):
            ctx.vjp(x, m, ab)
        elif a.pol in ("step", "step-comp"):
            ctx.run(x, v, m, a.steps)  # paper steps: pack + force sums with the kick/drift epilogue
        elif a.pol == "adjoint":
            ctx.adjoint(m, a.steps, ck, a.ckpt_every, xb, vb)
        else:
            ctx.energy(x, v, m)

    call()
    torch.cuda.synchronize()
    times = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    ctx.sync()
    t = min(times)
    inter = float(a.n) ** 2 * (a.steps if a.pol in ("step", "step-comp", "adjoint") else 1)
    print(json.dumps({"n": a.n, "pol": a.pol, "shape": ctx.get_config(a.n, mode), "s": t, "times": times,
                      "interactions_per_s": inter / t, "tflops_20": 20 * inter / t / 1e12}))


if __name__ == "__main__":
    main()
