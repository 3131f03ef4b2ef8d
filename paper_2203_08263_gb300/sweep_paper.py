"""The paper's workload sweep and math-operation ablation, on the GPU.

    python -m paper_2203_08263_gb300.sweep_paper --what sweep      # N = 256 ... 524288, I = 100
    python -m paper_2203_08263_gb300.sweep_paper --what ablation   # s^(3/2) variants

Sweep: for every N of the paper's Section 4.1 (powers of two from 256 to
524288) runs I = 100 steps of the printed update through nb_run, in FP32 and
in the precision form (FP64 state, compensated FP32 forces), each autotuned
for its size (kernel shape, and graph or one-cluster path), and reports
GFLOPS = 20 N^2 I / t, the paper's metric. Inputs: Plummer sphere (seed 1),
eps = 0.05, dt = 1e-3 (the paper does not state its initial conditions).

Ablation: the GPU analog of the paper's denominator experiment (Sections
3.2.6 and 3.3.6): MUFU rsqrt cubed, IEEE sqrt then division, and powf, each
timed on nb_accel and compared with the library's precision form (compensated
sums) on a subset of bodies; the parity tests hold the FP64 oracle.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

PAPER_N = [256 << k for k in range(12)]


def _timed(torch, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def sweep(steps: int, nmax: int):
    import torch

    from paper_2203_08263_gb300 import ics
    from paper_2203_08263_gb300.nbody import Context

    dev = torch.device("cuda:0")
    rows = []
    for n in [n for n in PAPER_N if n <= nmax]:
        s = ics.plummer(n, seed=1)
        row = {"n": n, "steps": steps}
        for prec, f in (("fp32", torch.float32), ("comp", torch.float64)):
            ctx = Context(1.0, 0.05, 1e-3, precision=prec)
            ctx.autotune(n)  # launch shape and nb_run path for this size
            x, v, m = (torch.tensor(a, dtype=f, device=dev) for a in (s.x, s.v, s.m))
            x0, v0 = x.clone(), v.clone()
            ctx.run(x, v, m, steps)  # the timed call once: its step graph is captured here
            x.copy_(x0)
            v.copy_(v0)
            t = _timed(torch, lambda: ctx.run(x, v, m, steps))
            ctx.sync()
            row[prec] = {"s": t, "gflops": 20.0 * n * n * steps / t / 1e9,
                         "interactions_per_s": float(n) * n * steps / t, "shape": ctx.get_config(n)}
            ctx.close()
        rows.append(row)
        print(json.dumps(row), flush=True)
    print("\n| N | FP32 GFLOPS (20 N^2 I / t) | precision form GFLOPS | FP32 s | precision form s |")
    print("|---|---|---|---|---|")
    for r in rows:
        print(f"| {r['n']} | {r['fp32']['gflops']:.0f} | {r['comp']['gflops']:.0f} | "
              f"{r['fp32']['s']:.4f} | {r['comp']['s']:.4f} |")


def ablation(n: int):
    import torch

    from paper_2203_08263_gb300 import ics
    from paper_2203_08263_gb300.nbody import NB_DBG_FORM, NB_DBG_MATH_VARIANT, Context

    dev = torch.device("cuda:0")
    s = ics.plummer(n, seed=1)
    idx = ics.subset_indices(n, 512, 9)
    x, m = (torch.tensor(a, dtype=torch.float32, device=dev) for a in (s.x, s.m))
    # reference: the library's precision form on the same FP32-rounded bodies
    # (compensated sums, about 3e-8 from an FP64 sum on this input class,
    # against the FP32 variants' 1e-7 .. 1e-6)
    comp = Context(1.0, 0.05, 1e-3, precision="comp")
    ref = comp.accel(x.double(), m.double()).cpu().numpy()[idx]
    comp.close()
    names = {0: "MUFU rsqrt, y^3", 1: "IEEE sqrt then division", 2: "powf(s, -1.5)",
             3: "MUFU rsqrt, y^3, pair-symmetric kernel"}
    print("\n| denominator | interactions/s | GFLOPS (20/interaction) | rel. L2 vs the precision form |")
    print("|---|---|---|---|")
    for var in (0, 1, 2, 3):
        ctx = Context(1.0, 0.05, 1e-3)
        # the three denominators on the one-sided kernels (the variants have
        # no pair-symmetric form); then the library's default kernel for n
        ctx.debug_set(NB_DBG_FORM, 0 if var == 3 else 1)
        ctx.debug_set(NB_DBG_MATH_VARIANT, 0 if var == 3 else var)
        a = ctx.accel(x, m)
        t = min(_timed(torch, lambda: ctx.accel(x, m)) for _ in range(3))
        err = float(np.linalg.norm(a.double().cpu().numpy()[idx] - ref) / np.linalg.norm(ref))
        rate = float(n) * n / t
        print(json.dumps({"variant": var, "name": names[var], "n": n, "s": t, "interactions_per_s": rate,
                          "rel_l2": err, "shape": ctx.get_config(n)}), flush=True)
        print(f"| {names[var]} | {rate:.3e} | {20 * rate / 1e9:.0f} | {err:.2e} |")
        ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--what", choices=["sweep", "ablation"], default="sweep")
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--nmax", type=int, default=524288)
    ap.add_argument("--n", type=int, default=65536)
    a = ap.parse_args()
    from paper_2203_08263_gb300 import build

    build.build()
    if a.what == "sweep":
        sweep(a.steps, a.nmax)
    else:
        ablation(a.n)


if __name__ == "__main__":
    main()
