"""GPU parity of nb_run's fused paths (every step in one kernel: the
one-cluster form with positions in distributed shared memory, and its grid
form exchanging positions through L2) against the FP64 oracle and against the
graph-of-launches path, through the C-ABI."""
import numpy as np
import pytest

import oracle
from paper_2203_08263_gb300 import ics
from gpu_util import ensure_built, rel_l2, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GRAPH, CLUSTER, GRID = 1, 2, 3


@pytest.fixture(scope="module")
def nbm():
    ensure_built()
    from paper_2203_08263_gb300 import nbody
    return nbody


def _t(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _ctx(nbm, path, G=1.0, eps=0.01, dt=1e-3, scheme="paper"):
    ctx = nbm.Context(G, eps, dt, scheme=scheme)
    ctx.debug_set(nbm.NB_DBG_RUN_PATH, path)
    return ctx


# odd sizes, slices that do not divide evenly, one body, and the paths' limits
@pytest.mark.parametrize("path,n", [(p, n) for p in (CLUSTER, GRID)
                                    for n in (1, 2, 3, 17, 255, 256, 1000, 1024, 2047, 3001, 4096)]
                         + [(GRID, 6001), (GRID, 8192)])
def test_cluster_run_matches_oracle(nbm, path, n):
    s = ics.cube(n, seed=500 + n)
    steps = 10
    ctx = _ctx(nbm, path)
    x, v, m = _t(s.x), _t(s.v), _t(s.m)
    before = ctx.launch_count
    ctx.run(x, v, m, steps)
    ctx.sync()
    # all steps in one kernel (the grid form's barrier counters reset themselves)
    assert ctx.launch_count - before == 1
    xr, vr = oracle.run(s.x, s.v, s.m, 1.0, 0.01, 1e-3, steps)
    assert rel_l2(to_np(x), xr) <= 1e-5
    assert rel_l2(to_np(v), vr) <= 1e-4


@pytest.mark.parametrize("path,n", [(CLUSTER, 64), (CLUSTER, 1500), (GRID, 64), (GRID, 5000)])
def test_cluster_run_kdk_matches_oracle(nbm, path, n):
    s = ics.cube(n, seed=900 + n)
    ctx = _ctx(nbm, path, G=0.8, eps=0.02, dt=2e-3, scheme="kdk")
    x, v, m = _t(s.x), _t(s.v), _t(s.m)
    ctx.run(x, v, m, 12)
    ctx.sync()
    xr, vr = oracle.run(s.x, s.v, s.m, 0.8, 0.02, 2e-3, 12, scheme="kdk")
    assert rel_l2(to_np(x), xr) <= 1e-5
    assert rel_l2(to_np(v), vr) <= 1e-4


@pytest.mark.parametrize("fused", [CLUSTER, GRID])
def test_cluster_and_graph_paths_agree_with_checkpoints(nbm, fused):
    n, steps, k = 777, 12, 4
    s = ics.cube(n, seed=31)
    out = {}
    for path in (GRAPH, fused):
        ctx = _ctx(nbm, path)
        x, v, m = _t(s.x), _t(s.v), _t(s.m)
        ck = torch.zeros((steps // k + 1, n, 6), dtype=torch.float32, device=DEV)
        ctx.run(x, v, m, steps, ckpt=ck, ckpt_every=k)
        ctx.sync()
        out[path] = (to_np(x), to_np(v), to_np(ck))
    xg, vg, cg = out[GRAPH]
    xc, vc, cc = out[fused]
    assert np.array_equal(cc[0][:, :3], s.x.astype(np.float32))  # slot 0 is the input state
    assert np.array_equal(cc[0][:, 3:], s.v.astype(np.float32))
    assert rel_l2(xc, xg) <= 1e-6 and rel_l2(vc, vg) <= 1e-5
    for slot in range(1, steps // k + 1):
        assert rel_l2(cc[slot], cg[slot]) <= 1e-5
    assert np.array_equal(cc[-1][:, :3], xc) and np.array_equal(cc[-1][:, 3:], vc)


def test_default_path_choice(nbm):
    """Untuned, FP32: the cluster path up to n = 512 (one launch for all
    steps), the grid form up to 4096 (one launch), the graph path above (the
    pack and one force launch per step)."""
    for n, launches in ((512, 1), (1024, 1), (4096, 1), (5000, 11)):
        s = ics.cube(n, seed=3)
        ctx = nbm.Context(1.0, 0.01, 1e-3)
        want = "cluster" if n <= 512 else ("grid" if n <= 4096 else "graph")
        rp = ctx.get_run_path(n)
        assert rp["path"] == want and not rp["tuned"], (n, rp)
        x, v, m = _t(s.x), _t(s.v), _t(s.m)
        ctx.run(x, v, m, 10)
        ctx.sync()
        before = ctx.launch_count
        ctx.run(x, v, m, 10)
        ctx.sync()
        assert ctx.launch_count - before == launches, n


def test_autotune_keeps_run_correct(nbm):
    n = 1024
    s = ics.cube(n, seed=0)
    ctx = nbm.Context(1.0, 0.01, 1e-3)
    ctx.autotune(n)
    assert ctx.get_run_path(n)["tuned"]
    x, v, m = _t(s.x), _t(s.v), _t(s.m)
    ctx.run(x, v, m, 10)
    ctx.sync()
    xr, _ = oracle.run(s.x, s.v, s.m, 1.0, 0.01, 1e-3, 10)
    assert rel_l2(to_np(x), xr) <= 1e-5


def test_cluster_path_refuses_what_it_cannot_run(nbm):
    s = ics.cube(5000, seed=1)
    ctx = _ctx(nbm, CLUSTER)
    with pytest.raises(RuntimeError):
        ctx.run(_t(s.x), _t(s.v), _t(s.m), 2)  # above 4096 bodies
    s = ics.cube(9000, seed=1)
    ctx = _ctx(nbm, GRID)
    with pytest.raises(RuntimeError):
        ctx.run(_t(s.x), _t(s.v), _t(s.m), 2)  # above 8192 bodies
    s = ics.cube(100, seed=1)
    ctx = _ctx(nbm, CLUSTER)
    ctx.debug_set(nbm.NB_DBG_MATH_VARIANT, 1)  # the sqrt-then-divide ablation has no cluster form
    with pytest.raises(RuntimeError):
        ctx.run(_t(s.x), _t(s.v), _t(s.m), 2)


# ---------------------------------------------------------- precision form

def _ctx64(nbm, path, G=1.0, eps=0.05, dt=5e-4, scheme="paper"):
    ctx = nbm.Context(G, eps, dt, precision="comp", scheme=scheme)
    ctx.debug_set(nbm.NB_DBG_RUN_PATH, path)
    return ctx


def _t64(a):
    return _t(a, torch.float64)


@pytest.mark.parametrize("path,n", [(CLUSTER, 3), (CLUSTER, 300), (CLUSTER, 2048), (CLUSTER, 4096),
                                    (GRID, 3), (GRID, 2048), (GRID, 8192)])
def test_cluster_precision_form_matches_oracle(nbm, path, n):
    """FP64 state, compensated FP32 forces: the tolerances of the graph
    path's precision-form run test (C3 setting, Plummer)."""
    s = ics.plummer(n, seed=2)
    ctx = _ctx64(nbm, path)
    x, v, m = _t64(s.x), _t64(s.v), _t64(s.m)
    ctx.run(x, v, m, 10)
    ctx.sync()
    xr, vr = oracle.run(s.x, s.v, s.m, 1.0, 0.05, 5e-4, 10)
    assert rel_l2(to_np(x), xr) <= 1e-9
    assert rel_l2(to_np(v), vr) <= 1e-6


def test_default_path_choice_precision_form(nbm):
    """Untuned, the precision form takes the cluster path up to n = 512, the
    grid form up to 8192 and the graph path above."""
    for n, launches in ((512, 1), (1024, 1), (8192, 1), (9000, 11)):
        s = ics.plummer(n, seed=5)
        ctx = nbm.Context(1.0, 0.05, 5e-4, precision="comp")
        x, v, m = _t64(s.x), _t64(s.v), _t64(s.m)
        ctx.run(x, v, m, 10)
        ctx.sync()
        before = ctx.launch_count
        ctx.run(x, v, m, 10)
        ctx.sync()
        assert ctx.launch_count - before == launches, n


def test_cluster_precision_form_kdk_and_checkpoints(nbm):
    n = 1000
    s = ics.plummer(n, seed=12)
    ctx = _ctx64(nbm, CLUSTER, scheme="kdk")
    x, v, m = _t64(s.x), _t64(s.v), _t64(s.m)
    ctx.run(x, v, m, 8)
    ctx.sync()
    xr, vr = oracle.run(s.x, s.v, s.m, 1.0, 0.05, 5e-4, 8, scheme="kdk")
    assert rel_l2(to_np(x), xr) <= 1e-9 and rel_l2(to_np(v), vr) <= 1e-6
    out = {}
    for path in (GRAPH, CLUSTER):
        ctx = _ctx64(nbm, path)
        x, v, m = _t64(s.x), _t64(s.v), _t64(s.m)
        ck = torch.zeros((3, n, 6), dtype=torch.float64, device=DEV)
        ctx.run(x, v, m, 8, ckpt=ck, ckpt_every=4)
        ctx.sync()
        out[path] = to_np(ck)
    assert np.array_equal(out[CLUSTER][0], out[GRAPH][0])  # the input state, exactly
    for slot in (1, 2):
        assert rel_l2(out[CLUSTER][slot], out[GRAPH][slot]) <= 1e-9


def test_grid_barrier_timeout_is_reported(nbm):
    """With CTA 0 held back from the grid barrier (a debug flag) every
    barrier wait of the grid form runs out after 1 ms: the kernel ends, and
    nb_sync reports the timeout; the context then runs correctly again."""
    n = 4096
    s = ics.cube(n, seed=77)
    ctx = _ctx(nbm, GRID)
    x, v, m = _t(s.x), _t(s.v), _t(s.m)
    ctx.debug_set(nbm.NB_DBG_WAIT_TIMEOUT_NS, 1_000_000)
    ctx.debug_set(nbm.NB_DBG_STALL_PRODUCER, 1)
    ctx.run(x, v, m, 50)
    with pytest.raises(RuntimeError):
        ctx.sync()
    ctx.debug_set(nbm.NB_DBG_STALL_PRODUCER, 0)
    ctx.debug_set(nbm.NB_DBG_WAIT_TIMEOUT_NS, 2_000_000_000)
    x, v = _t(s.x), _t(s.v)
    ctx.run(x, v, m, 5)
    ctx.sync()
    xr, _ = oracle.run(s.x, s.v, s.m, 1.0, 0.01, 1e-3, 5)
    assert rel_l2(to_np(x), xr) <= 1e-5
