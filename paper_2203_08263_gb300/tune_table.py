"""Write the autotuner's table for this GPU type.

    python -m paper_2203_08263_gb300.tune_table [--out PATH] [--only fp32|comp]

Runs nb_autotune for the problem sizes of the library's standard workloads
(FP32 forces, FP32 VJP, precision-form forces and VJP) and lets the library
store the winners in a JSON file (the format NB_AUTOTUNE_CACHE reads). The
default output is tuned/<device name>.json inside the package, which
bench.py loads so that its launch shapes are the tuner's and reproducible.
"""
from __future__ import annotations

import argparse
import os

HERE = os.path.dirname(os.path.abspath(__file__))

FP32_FORWARD = [256, 512, 1024, 2048, 4096, 8192, 16384, 32768, 65536, 131072, 262144, 524288]
FP32_ADJOINT = [2048, 16384]
COMP_FORWARD = [256, 512, 1024, 2048, 4096, 8192, 16384, 65536, 262144, 1048576]
COMP_ADJOINT = [2048, 16384]


def table_path(device_name: str) -> str:
    slug = "".join(c if c.isalnum() else "_" for c in device_name)
    return os.path.join(HERE, "tuned", f"{slug}.json")


def main():
    import torch

    from paper_2203_08263_gb300 import build

    build.build()
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--only", default="all", choices=["all", "fp32", "comp"],
                    help="retune one precision and keep the table's other entries")
    a = ap.parse_args()
    out = a.out or table_path(torch.cuda.get_device_name(0))
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if os.path.exists(out) and a.only == "all":
        os.unlink(out)
    os.environ["NB_AUTOTUNE_CACHE"] = out  # read at context creation, written by each tune
    from paper_2203_08263_gb300.nbody import MODE_ADJOINT, MODE_FORWARD, Context

    if a.only in ("all", "fp32"):
        ctx = Context(1.0, 0.05, 1e-3)
        for n in FP32_FORWARD:
            ctx.autotune(n, MODE_FORWARD)
            print("fp32 forward", n, ctx.get_config(n, MODE_FORWARD), flush=True)
        for n in FP32_ADJOINT:
            ctx.autotune(n, MODE_ADJOINT)
            print("fp32 adjoint", n, ctx.get_config(n, MODE_ADJOINT), flush=True)
        ctx.close()
    if a.only in ("all", "comp"):
        ctx = Context(1.0, 0.05, 1e-3, precision="comp")  # loads the FP32 entries, adds its own
        for n in COMP_FORWARD:
            ctx.autotune(n, MODE_FORWARD)
            print("comp forward", n, ctx.get_config(n, MODE_FORWARD), flush=True)
        for n in COMP_ADJOINT:
            ctx.autotune(n, MODE_ADJOINT)
            print("comp adjoint", n, ctx.get_config(n, MODE_ADJOINT), flush=True)
        ctx.close()
    print("wrote", out)


if __name__ == "__main__":
    main()
