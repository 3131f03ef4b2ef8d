"""Thin Python binding of libnbody (include/nbody.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels. The module-level ``nb_*`` functions mirror the C-ABI one to one;
:class:`Context` wraps them for torch tensors (device memory and streams come
from PyTorch). Nothing here computes forces, and there is no CPU fallback: if
``libnbody.so`` is missing or cannot load, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libnbody.so")

NB_OK, NB_ERR_INVALID, NB_ERR_CUDA, NB_ERR_NOMEM, NB_ERR_TIMEOUT, NB_ERR_UNSUPPORTED = range(6)
NB_FP32, NB_FP32_COMP_FP64_STATE = 0, 1
NB_SCHEME_PAPER, NB_SCHEME_KDK = 0, 1
NB_DBG_WAIT_TIMEOUT_NS, NB_DBG_STALL_PRODUCER, NB_DBG_MATH_VARIANT, NB_DBG_RUN_PATH = 1, 2, 3, 4
NB_DBG_FORM, NB_DBG_VJP_FORM, NB_DBG_SYM_TILE, NB_DBG_ADJ_PREP = 5, 6, 7, 8
MODE_FORWARD, MODE_ADJOINT, MODE_POTENTIAL = 0, 1, 2
# nb_form values (nb_get_form)
FORMS = {0: "f32x2", 1: "scalar", 2: "compensated", 3: "potential", 4: "vjp",
         5: "vjp_compensated", 6: "sqrt_div", 7: "pow", 8: "pair_symmetric", 9: "vjp_pair_symmetric",
         10: "compensated_pair_symmetric", 11: "vjp_compensated_pair_symmetric"}

# Every symbol include/nbody.h declares, with (restype, argtypes).
_c = ctypes
_vp, _i64, _i, _d = _c.c_void_p, _c.c_int64, _c.c_int, _c.c_double


class nb_params(ctypes.Structure):
    _fields_ = [("G", _d), ("eps", _d), ("dt", _d), ("precision", _i), ("scheme", _i),
                ("tile_override", _i * 4)]


SIGNATURES = {
    "nb_abi_version": (_i, []),
    "nb_create": (_i, [_c.POINTER(_vp), _i, _c.POINTER(nb_params)]),
    "nb_destroy": (None, [_vp]),
    "nb_status_string": (_c.c_char_p, [_i]),
    "nb_last_error": (_c.c_char_p, [_vp]),
    "nb_set_params": (_i, [_vp, _d, _d, _d]),
    "nb_accel": (_i, [_vp, _i64, _vp, _vp, _vp, _vp]),
    "nb_step": (_i, [_vp, _i64, _vp, _vp, _vp, _vp]),
    "nb_run": (_i, [_vp, _i64, _vp, _vp, _vp, _i, _vp, _i, _vp]),
    "nb_run_batched": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _i, _vp]),
    "nb_batched_max_n": (_i64, []),
    "nb_autotune_batched": (_i, [_vp, _i, _vp]),
    "nb_get_batched_config": (_i, [_vp, _i, _vp, _c.POINTER(_i)]),
    "nb_set_batched_config": (_i, [_vp, _i, _vp, _i, _i, _i]),
    "nb_set_batched_form": (_i, [_vp, _i, _vp, _i]),
    "nb_get_batched_form": (_i, [_vp, _i, _vp, _c.POINTER(_i)]),
    "nb_get_run_path": (_i, [_vp, _i64, _c.POINTER(_i)]),
    "nb_adjoint": (_i, [_vp, _i64, _vp, _i, _vp, _i, _vp, _vp, _vp, _vp, _vp, _vp]),
    "nb_vjp": (_i, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "nb_energy": (_i, [_vp, _i64, _vp, _vp, _vp, _c.POINTER(_d), _vp]),
    "nb_autotune": (_i, [_vp, _i64, _i]),
    "nb_get_config": (_i, [_vp, _i64, _i, _c.POINTER(_i)]),
    "nb_get_form": (_i, [_vp, _i64, _i, _c.POINTER(_i)]),
    "nb_sync": (_i, [_vp, _vp]),
    "nb_launch_count": (_i64, [_vp]),
    "nb_debug_set": (_i, [_vp, _i, _i64]),
    "nb_measure_peaks": (_i, [_vp, _c.POINTER(_d)]),
    "nb_accel_noalloc": (_i, [_i64, _vp, _vp, _vp, _d, _d, _vp]),
}
NB_NOALLOC_MAX_N = 32768

_lock = threading.Lock()
_lib = None


class NBodyError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


def load(path: str | None = None):
    """Load libnbody.so (built by ``paper_2203_08263_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise NBodyError(NB_ERR_UNSUPPORTED,
                             f"libnbody.so not found at {p}: run paper_2203_08263_gb300.build.build()")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if lib.nb_abi_version() != 1:
            raise NBodyError(NB_ERR_UNSUPPORTED, "libnbody ABI version mismatch")
        if path is None:
            _lib = lib
        return lib


def __getattr__(name):
    # module-level nb_* names forward to the C functions of the same name
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)


# ------------------------------------------------------------------ helpers

def _torch():
    import torch
    return torch


def _ptr(a) -> int:
    """Address of a contiguous torch tensor or numpy array."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr()


def _stream(stream, device) -> int:
    torch = _torch()
    if stream is None:
        return torch.cuda.current_stream(device).cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Context:
    """A libnbody context: parameters, scratch memory, graphs, tuning table."""

    def __init__(self, G: float, eps: float, dt: float, precision: str = "fp32",
                 scheme: str = "paper", device: int | None = None, tile_override=None):
        torch = _torch()
        self.lib = load()
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.precision = {"fp32": NB_FP32, "comp": NB_FP32_COMP_FP64_STATE}[precision]
        self.dtype = torch.float32 if self.precision == NB_FP32 else torch.float64
        p = nb_params(G, eps, dt, self.precision,
                      {"paper": NB_SCHEME_PAPER, "kdk": NB_SCHEME_KDK}[scheme],
                      (_i * 4)(*(tile_override or (0, 0, 0, 0))))
        h = _vp()
        st = self.lib.nb_create(ctypes.byref(h), self.device, ctypes.byref(p))
        if st != NB_OK:
            raise NBodyError(st, f"nb_create: {self.lib.nb_status_string(st).decode()}")
        self.h = h
        self.G, self.eps, self.dt = G, eps, dt

    def close(self):
        if getattr(self, "h", None):
            self.lib.nb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st != NB_OK:
            msg = self.lib.nb_last_error(self.h).decode()
            raise NBodyError(st, f"{what}: {self.lib.nb_status_string(st).decode()}: {msg}")

    def _s(self, stream):
        return _stream(stream, self.device)

    def set_params(self, G, eps, dt):
        self._check(self.lib.nb_set_params(self.h, G, eps, dt), "nb_set_params")
        self.G, self.eps, self.dt = G, eps, dt

    # ---- forward
    def accel(self, x, m, out=None, stream=None):
        torch = _torch()
        n = int(m.shape[0])
        if out is None:
            out = torch.empty((n, 3), dtype=x.dtype, device=x.device) if not isinstance(x, np.ndarray) \
                else np.empty((n, 3), dtype=x.dtype)
        self._check(self.lib.nb_accel(self.h, n, _ptr(x), _ptr(m), _ptr(out), self._s(stream)), "nb_accel")
        return out

    def step(self, x, v, m, stream=None):
        self._check(self.lib.nb_step(self.h, int(m.shape[0]), _ptr(x), _ptr(v), _ptr(m), self._s(stream)),
                    "nb_step")

    def run(self, x, v, m, steps: int, ckpt=None, ckpt_every: int = 0, stream=None):
        self._check(self.lib.nb_run(self.h, int(m.shape[0]), _ptr(x), _ptr(v), _ptr(m), int(steps),
                                    _ptr(ckpt) if ckpt is not None else None, int(ckpt_every),
                                    self._s(stream)), "nb_run")

    def run_batched(self, offsets, x, v, m, steps: int, stream=None):
        nsys = int(offsets.shape[0]) - 1
        self._check(self.lib.nb_run_batched(self.h, nsys, _ptr(offsets), _ptr(x), _ptr(v), _ptr(m),
                                            int(steps), self._s(stream)), "nb_run_batched")

    def autotune_batched(self, offsets):
        self._check(self.lib.nb_autotune_batched(self.h, int(offsets.shape[0]) - 1, _ptr(offsets)),
                    "nb_autotune_batched")

    def get_batched_config(self, offsets) -> dict:
        out = (_i * 6)()
        self._check(self.lib.nb_get_batched_config(self.h, int(offsets.shape[0]) - 1, _ptr(offsets), out),
                    "nb_get_batched_config")
        form = _i()
        self._check(self.lib.nb_get_batched_form(self.h, int(offsets.shape[0]) - 1, _ptr(offsets),
                                                 ctypes.byref(form)), "nb_get_batched_form")
        return {"threads": out[0], "bodies_per_thread": out[1], "jtile": out[2], "items_per_step": out[3],
                "ctas": out[4], "tuned": out[5] == 1, "pinned": out[5] == 2,
                "form": {1: "one_sided", 2: "pair_symmetric"}[form.value]}

    def set_batched_form(self, offsets, form: str | None):
        """Pin the batched form for these sizes ("one_sided", "pair_symmetric"); None clears."""
        f = {None: 0, "one_sided": 1, "pair_symmetric": 2}[form]
        self._check(self.lib.nb_set_batched_form(self.h, int(offsets.shape[0]) - 1, _ptr(offsets), f),
                    "nb_set_batched_form")

    def get_run_path(self, n: int) -> dict:
        """The nb_run path for n bodies: graph, cluster or grid, its size, and whether it was tuned."""
        out = (_i * 3)()
        self._check(self.lib.nb_get_run_path(self.h, int(n), out), "nb_get_run_path")
        return {"path": {1: "graph", 2: "cluster", 3: "grid"}[out[0]], "size": out[1], "tuned": bool(out[2])}

    def set_batched_config(self, offsets, threads: int, bodies_per_thread: int, jtile: int):
        """Pin the batched shape for these sizes; (0, 0, 0) returns to the default."""
        self._check(self.lib.nb_set_batched_config(self.h, int(offsets.shape[0]) - 1, _ptr(offsets),
                                                   int(threads), int(bodies_per_thread), int(jtile)),
                    "nb_set_batched_config")

    # ---- reverse
    def vjp(self, x, m, abar, stream=None):
        torch = _torch()
        n = int(m.shape[0])
        xbar = torch.empty((n, 3), dtype=x.dtype, device=x.device)
        mbar = torch.empty((n,), dtype=x.dtype, device=x.device)
        self._check(self.lib.nb_vjp(self.h, n, _ptr(x), _ptr(m), _ptr(abar), _ptr(xbar), _ptr(mbar),
                                    self._s(stream)), "nb_vjp")
        return xbar, mbar

    def adjoint(self, m, steps, ckpt, ckpt_every, xbar_T, vbar_T, stream=None):
        torch = _torch()
        n = int(m.shape[0])
        xbar0 = torch.empty((n, 3), dtype=m.dtype, device=m.device)
        vbar0 = torch.empty((n, 3), dtype=m.dtype, device=m.device)
        mbar = torch.empty((n,), dtype=m.dtype, device=m.device)
        self._check(self.lib.nb_adjoint(self.h, n, _ptr(m), int(steps), _ptr(ckpt), int(ckpt_every),
                                        _ptr(xbar_T), _ptr(vbar_T), _ptr(xbar0), _ptr(vbar0), _ptr(mbar),
                                        self._s(stream)), "nb_adjoint")
        return xbar0, vbar0, mbar

    # ---- diagnostics, tuning, control
    def energy(self, x, v, m, stream=None) -> dict:
        out = (_d * 6)()
        self._check(self.lib.nb_energy(self.h, int(m.shape[0]), _ptr(x), _ptr(v), _ptr(m), out,
                                       self._s(stream)), "nb_energy")
        return {"P": np.array(out[0:3]), "KE": out[3], "Phi": out[4], "H": out[5]}

    def autotune(self, n: int, mode: int = MODE_FORWARD):
        self._check(self.lib.nb_autotune(self.h, int(n), int(mode)), "nb_autotune")

    def get_config(self, n: int, mode: int = MODE_FORWARD) -> dict:
        out = (_i * 5)()
        self._check(self.lib.nb_get_config(self.h, int(n), int(mode), out), "nb_get_config")
        form = _i()
        self._check(self.lib.nb_get_form(self.h, int(n), int(mode), ctypes.byref(form)), "nb_get_form")
        return {"threads": out[0], "bodies_per_thread": out[1], "split": out[2], "jtile": out[3],
                "tuned": bool(out[4]), "form": FORMS.get(form.value, str(form.value))}

    def sync(self, stream=None):
        self._check(self.lib.nb_sync(self.h, self._s(stream)), "nb_sync")

    @property
    def launch_count(self) -> int:
        return int(self.lib.nb_launch_count(self.h))

    def measure_peaks(self) -> dict:
        out = (_d * 3)()
        self._check(self.lib.nb_measure_peaks(self.h, out), "nb_measure_peaks")
        return {"ffma_tflops": out[0], "ffma2_tflops": out[1], "mufu_rsqrt_gops": out[2]}

    def debug_set(self, key: int, value: int):
        self._check(self.lib.nb_debug_set(self.h, int(key), int(value)), "nb_debug_set")
