"""FP64 CPU oracle for the all-pairs N-body step (test infrastructure).

This package is the independent, plain definition that the CUDA library is
checked against. Only the tests, the smoke check and the benchmark's CPU
baseline may import it; the library itself never does, and the two share no
code. The arithmetic lives in ``nbody_oracle.c`` (IEEE double, OpenMP static
schedule over the output index, no fast-math, no FMA contraction); this module
only builds it with gcc and marshals numpy arrays.

Function map (paper = Milla & Rucci, arXiv 2203.08263):
  accel   -- Section 2.3 force sum, the inner j-loop of the Section 3.2.4 and
             3.3.5 figures: a_i = G sum_j m_j d_ij / (|d_ij|^2 + eps^2)^(3/2)
  step/run -- the printed update: half kick v += a dt/2, then x += v dt with
             the new v, all accelerations from the old positions
  run_kdk -- velocity Verlet, named (not printed) in Sections 3.2.3 and 3.3.7
  energy  -- momentum, kinetic energy, softened potential and H' = KE + Phi/2
  vjp / adjoint -- reverse mode of the above, Jacobian blocks written out
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nbody_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile nbody_oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i64, d, ci = ctypes.c_int64, ctypes.c_double, ctypes.c_int
        lib.oracle_accel.argtypes = [i64, dp, dp, d, d, i64, i64p, dp]
        lib.oracle_accel.restype = None
        for name in ("oracle_step",):
            getattr(lib, name).argtypes = [i64, dp, dp, dp, d, d, d]
            getattr(lib, name).restype = ci
        for name in ("oracle_run", "oracle_run_kdk"):
            getattr(lib, name).argtypes = [i64, dp, dp, dp, d, d, d, ci]
            getattr(lib, name).restype = ci
        lib.oracle_energy.argtypes = [i64, dp, dp, dp, d, d, dp]
        lib.oracle_energy.restype = None
        lib.oracle_vjp.argtypes = [i64, dp, dp, d, d, dp, dp, dp]
        lib.oracle_vjp.restype = None
        lib.oracle_adjoint.argtypes = [i64, dp, dp, dp, d, d, d, ci, dp, dp, dp, dp, dp]
        lib.oracle_adjoint.restype = ci
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ci
        lib.oracle_set_num_threads.argtypes = [ci]
        lib.oracle_set_num_threads.restype = None
        _lib = lib
        return lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(t: int) -> None:
    _load().oracle_set_num_threads(int(t))


def accel(x, m, G: float, eps: float, idx=None) -> np.ndarray:
    """a_i for every i (idx None) or for i in idx; returns (len, 3) float64."""
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    lib = _load()
    if idx is None:
        out = np.zeros((n, 3))
        lib.oracle_accel(n, _p(x), _p(m), G, eps, n, None, _p(out))
    else:
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
        if idx.size and (idx.min() < 0 or idx.max() >= n):
            raise IndexError("subset index out of range")
        out = np.zeros((idx.shape[0], 3))
        lib.oracle_accel(n, _p(x), _p(m), G, eps, idx.shape[0],
                         idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _p(out))
    return out


def run(x, v, m, G: float, eps: float, dt: float, steps: int, scheme: str = "paper"):
    """Returns (x, v) after `steps` updates; inputs are not modified."""
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3)).copy()
    v = _f64(v, (n, 3)).copy()
    lib = _load()
    fn = lib.oracle_run if scheme == "paper" else lib.oracle_run_kdk
    if scheme not in ("paper", "kdk"):
        raise ValueError(scheme)
    if fn(n, _p(x), _p(v), _p(m), G, eps, dt, int(steps)) != 0:
        raise MemoryError("oracle_run")
    return x, v


def step(x, v, m, G: float, eps: float, dt: float):
    return run(x, v, m, G, eps, dt, 1)


def energy(x, v, m, G: float, eps: float) -> dict:
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    v = _f64(v, (n, 3))
    out = np.zeros(6)
    _load().oracle_energy(n, _p(x), _p(v), _p(m), G, eps, _p(out))
    return {"P": out[0:3].copy(), "KE": out[3], "Phi": out[4], "H": out[5]}


def vjp(x, m, G: float, eps: float, abar):
    """(xbar, mbar) = abar^T da/dx, abar^T da/dm at positions x."""
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    abar = _f64(abar, (n, 3))
    xbar = np.zeros((n, 3))
    mbar = np.zeros(n)
    _load().oracle_vjp(n, _p(x), _p(m), G, eps, _p(abar), _p(xbar), _p(mbar))
    return xbar, mbar


def adjoint(x0, v0, m, G: float, eps: float, dt: float, steps: int, xbar_T, vbar_T):
    """Gradients (xbar0, vbar0, mbar) of a loss with cotangents (xbar_T, vbar_T)
    at the final state of `steps` paper updates from (x0, v0)."""
    m = _f64(m)
    n = m.shape[0]
    x0 = _f64(x0, (n, 3))
    v0 = _f64(v0, (n, 3))
    xbT = _f64(xbar_T, (n, 3))
    vbT = _f64(vbar_T, (n, 3))
    xb = np.zeros((n, 3))
    vb = np.zeros((n, 3))
    mb = np.zeros(n)
    rc = _load().oracle_adjoint(n, _p(x0), _p(v0), _p(m), G, eps, dt, int(steps),
                                _p(xbT), _p(vbT), _p(xb), _p(vb), _p(mb))
    if rc != 0:
        raise MemoryError("oracle_adjoint")
    return xb, vb, mb
