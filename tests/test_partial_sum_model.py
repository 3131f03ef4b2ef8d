"""CPU model of the summation orders of the force kernels (FP32 pair terms
summed in FP32 runs, the runs combined exactly, as the two-sum epilogues of
the precision form do): the error of runs as long as the pair-symmetric
kernels' (up to 512 terms per half-sum) stays far inside the compensated
form's 1e-6 bound on close-encounter-heavy input. numpy only; no oracle, no
GPU."""
import numpy as np

from paper_2203_08263_gb300 import ics


def _terms(n, eps, seed):
    s = ics.cube(n, seed=seed)
    x = s.x.astype(np.float32)
    m = s.m.astype(np.float32)
    e2 = np.float32(eps * eps)
    d = (x[None, :, :] - x[:, None, :]).astype(np.float32)
    q = (d[..., 0] * d[..., 0] + e2).astype(np.float32)
    q = (d[..., 1] * d[..., 1] + q).astype(np.float32)
    q = (d[..., 2] * d[..., 2] + q).astype(np.float32)
    y = (1.0 / np.sqrt(q.astype(np.float64))).astype(np.float32)  # a correctly rounded rsqrt
    y3 = ((y * y).astype(np.float32) * y).astype(np.float32)
    w = (m[None, :] * y3).astype(np.float32)
    t = (w[..., None] * d).astype(np.float32)
    xd = x.astype(np.float64)
    dd = xd[None, :, :] - xd[:, None, :]
    r2 = (dd ** 2).sum(-1) + float(e2)
    exact = (m.astype(np.float64)[None, :, None] * dd / r2[..., None] ** 1.5).sum(1)
    return t, exact


def _runs(t, length):
    out = np.zeros((t.shape[0], 3))
    for a in range(0, t.shape[1], length):
        acc = np.zeros((t.shape[0], 3), np.float32)
        for j in range(a, min(a + length, t.shape[1])):
            acc = (acc + t[:, j, :]).astype(np.float32)
        out += acc
    return out


def test_long_fp32_partials_within_compensated_bound():
    t, exact = _terms(1024, 0.01, seed=7)
    errs = {}
    for length in (32, 512, 1024):
        got = _runs(t, length)
        errs[length] = np.linalg.norm(got - exact) / np.linalg.norm(exact)
    assert errs[512] <= 1e-6 and errs[1024] <= 1e-6, errs
    assert errs[32] <= errs[1024]  # longer FP32 runs do not help
