"""Build libnbody.so from csrc/ with nvcc for sm_103a (in-tree, parallel).

Objects and the library go to paper_2203_08263_gb300/_build/. Rebuilds only
what changed (any header change rebuilds everything).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libnbody.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]
# extra nvcc flags (e.g. -DNB_JP_UNROLL=4); a change of flags rebuilds everything
EXTRA = os.environ.get("NB_NVCC_FLAGS", "").split()


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnbody")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    hs += glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(h) for h in hs)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(os.path.join(OUT, "obj"), exist_ok=True)
    stamp = os.path.join(OUT, "flags.txt")
    flags_now = " ".join(ARCH + FLAGS + EXTRA)
    if not os.path.exists(stamp) or open(stamp).read() != flags_now:
        force = True
    hm = _headers_mtime()
    cc = nvcc()
    jobs = []
    objs = []
    for src in sources():
        obj = os.path.join(OUT, "obj", os.path.basename(src) + ".o")
        objs.append(obj)
        if (force or not os.path.exists(obj) or os.path.getmtime(obj) < max(hm, os.path.getmtime(src))):
            jobs.append([cc, *ARCH, *FLAGS, *EXTRA, "-c", src, "-o", obj])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
            for j, f in zip(jobs, futs):
                r = f.result()
                if verbose and r.stdout:
                    print(r.stdout)
                if r.returncode != 0:
                    raise RuntimeError(f"nvcc failed for {j[-3]}:\n{r.stderr}")
    if jobs or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        r = subprocess.run([cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(flags_now)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
