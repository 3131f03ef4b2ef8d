"""nb_accel_noalloc, the allocation-free force sum, against nb_accel.

Callers that cannot allocate device memory when they need forces (inside a
stream capture, under a pooling allocator, or with a footprint fixed at load
time) use this entry point; it works from a static device array instead of
context scratch. This file is collected last so that a failure here leaves
every other test already run; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

from paper_2203_08263_gb300 import ics
from gpu_util import ensure_built, rel_l2, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_matches_nb_accel_on_two_calls_in_a_row():
    ensure_built()
    from paper_2203_08263_gb300 import nbody

    lib = nbody.load()
    G, eps = 1.0, 0.01
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    ctx = nbody.Context(G, eps, 1e-3, device=0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    cases = []
    for n, seed in ((3001, 1), (nbody.NB_NOALLOC_MAX_N, 2)):
        s = ics.cube(n, seed=seed)
        x = torch.tensor(s.x, dtype=torch.float32, device=dev)
        m = torch.tensor(s.m, dtype=torch.float32, device=dev)
        cases.append((n, x, m, torch.full((n, 3), float("nan"), device=dev)))
    # two calls back to back on one stream, then compare both results
    for n, x, m, a in cases:
        st = lib.nb_accel_noalloc(n, x.data_ptr(), m.data_ptr(), a.data_ptr(), G, eps, stream)
        assert st == nbody.NB_OK
    torch.cuda.synchronize()
    for n, x, m, a in cases:
        ref = to_np(ctx.accel(x, m))
        assert np.isfinite(to_np(a)).all()
        assert rel_l2(to_np(a), ref) <= 2e-5
    # sizes beyond the static array are refused before any launch
    n, x, m, a = cases[-1]
    assert lib.nb_accel_noalloc(nbody.NB_NOALLOC_MAX_N + 1, x.data_ptr(), m.data_ptr(), a.data_ptr(),
                                G, eps, stream) == nbody.NB_ERR_INVALID
    assert lib.nb_accel_noalloc(10, x.data_ptr(), m.data_ptr(), a.data_ptr(), G, 0.0,
                                stream) == nbody.NB_ERR_INVALID
    ctx.close()
