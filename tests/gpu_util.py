"""Shared helpers for the GPU parity tests (inputs, error metric)."""
import numpy as np

from paper_2203_08263_gb300 import build as nbuild


def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def to_np(t):
    return t.detach().double().cpu().numpy()


_built = False


def ensure_built():
    global _built
    if not _built:
        nbuild.build()
        _built = True
