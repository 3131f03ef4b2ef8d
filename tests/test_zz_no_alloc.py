"""nb_accel_noalloc, the allocation-free force sum, against the FP64 oracle
and against nb_accel.

Callers that cannot allocate device memory when they need forces (a process
whose device memory belongs to a pooling allocator, or a service whose
footprint is fixed when the library loads) use this entry point; it works
from a static device array instead of context scratch. This file is collected
last so that a failure here leaves every other test already run; it passes
alone in a fresh process as well.
"""
import numpy as np
import pytest

import oracle
from paper_2203_08263_gb300 import ics
from gpu_util import ensure_built, rel_l2, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_matches_oracle_on_two_calls_in_a_row():
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
        cases.append((s, x, m, torch.full((n, 3), float("nan"), device=dev)))
    # two calls back to back on one stream (the second reuses the static
    # array the first one filled), then compare both results
    for s, x, m, a in cases:
        st = lib.nb_accel_noalloc(s.n, x.data_ptr(), m.data_ptr(), a.data_ptr(), G, eps, stream)
        assert st == nbody.NB_OK
    torch.cuda.synchronize()
    for s, x, m, a in cases:
        got = to_np(a)
        assert np.isfinite(got).all()
        idx = ics.subset_indices(s.n, 1024, 5)
        assert rel_l2(got[idx], oracle.accel(s.x, s.m, G, eps, idx)) <= 2e-5
        assert rel_l2(got, to_np(ctx.accel(x, m))) <= 2e-5

    # argument errors are refused on the host, before any launch
    s, x, m, a = cases[0]
    n = s.n
    assert lib.nb_accel_noalloc(nbody.NB_NOALLOC_MAX_N + 1, x.data_ptr(), m.data_ptr(), a.data_ptr(),
                                G, eps, stream) == nbody.NB_ERR_INVALID
    assert lib.nb_accel_noalloc(10, x.data_ptr(), m.data_ptr(), a.data_ptr(), G, 0.0,
                                stream) == nbody.NB_ERR_INVALID
    host = np.zeros((n, 3), dtype=np.float32)
    assert lib.nb_accel_noalloc(n, host.ctypes.data, m.data_ptr(), a.data_ptr(), G, eps,
                                stream) == nbody.NB_ERR_INVALID
    assert lib.nb_accel_noalloc(n, x.data_ptr(), m.data_ptr(), host.ctypes.data, G, eps,
                                stream) == nbody.NB_ERR_INVALID
    assert lib.nb_accel_noalloc(n - 1, x.data_ptr() + 2, m.data_ptr(), a.data_ptr(), G, eps,
                                stream) == nbody.NB_ERR_INVALID
    assert lib.nb_accel_noalloc(n, x.data_ptr(), None, a.data_ptr(), G, eps,
                                stream) == nbody.NB_ERR_INVALID
    # the refused calls wrote nothing: the last result is still the first case's
    torch.cuda.synchronize()
    idx = ics.subset_indices(n, 1024, 5)
    assert rel_l2(to_np(a)[idx], oracle.accel(s.x, s.m, G, eps, idx)) <= 2e-5
    ctx.close()
