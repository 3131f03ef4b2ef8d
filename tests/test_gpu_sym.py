"""GPU parity of the pair-symmetric FP32 kernels (each unordered pair once,
its terms added to both bodies) against the FP64 oracle, through the C-ABI:
accelerations (<= 2e-5 relative L2), runs of both update schemes,
checkpoints, determinism, the adjoint VJP (<= 5e-5) and whole adjoints, and
the padding of the step buffers."""
import numpy as np
import pytest

import oracle
from paper_2203_08263_gb300 import ics
from gpu_util import ensure_built, rel_l2, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GRAPH = 1


@pytest.fixture(scope="module")
def nbm():
    ensure_built()
    from paper_2203_08263_gb300 import nbody
    return nbody


def _t(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _ctx(nbm, block, G=1.0, eps=0.01, dt=1e-3, scheme="paper"):
    ctx = nbm.Context(G, eps, dt, scheme=scheme)
    ctx.debug_set(nbm.NB_DBG_FORM, block)
    ctx.debug_set(nbm.NB_DBG_RUN_PATH, GRAPH)
    return ctx


# one body (the diagonal item alone), odd sizes, one and several blocks with
# ragged padding, exact multiples of the block
@pytest.mark.parametrize("block", [256, 512, 1024])
@pytest.mark.parametrize("n", [1, 2, 3, 63, 64, 65, 255, 257, 511, 512, 513, 1000, 1024, 2047, 3001, 5120])
def test_sym_accel_matches_oracle(nbm, block, n):
    G, eps = 0.9, 0.02
    s = ics.cube(n, seed=300 + n)
    ctx = _ctx(nbm, block, G, eps)
    assert ctx.get_config(n)["form"] == "pair_symmetric"
    a = to_np(ctx.accel(_t(s.x), _t(s.m)))
    ref = oracle.accel(s.x, s.m, G, eps)
    if n == 1:
        assert np.all(a == 0.0)
    else:
        assert rel_l2(a, ref) <= 2e-5


def test_sym_split_blocks_match_oracle(nbm):
    """Blocks of 256 bodies whose block pairs two warps share, each taking
    half of the j-chunks (the untuned choice from 16384 to 32767 bodies): a
    ragged size (17000 bodies, 67 blocks) against the oracle in both
    precisions and over a KDK run, bit-identical by tiles and on a repeat."""
    n, G, eps, dt = 17000, 1.0, 0.01, 1e-3
    s = ics.cube(n, seed=77)
    ctx = nbm.Context(G, eps, dt)
    if ctx.get_config(n)["tuned"]:
        pytest.skip("a tuning table is loaded")
    cfg = ctx.get_config(n)
    assert (cfg["form"], cfg["threads"], cfg["bodies_per_thread"]) == ("pair_symmetric", 64, 4)
    ref = oracle.accel(s.x, s.m, G, eps)
    a = ctx.accel(_t(s.x), _t(s.m))
    assert rel_l2(to_np(a), ref) <= 2e-5
    assert torch.equal(ctx.accel(_t(s.x), _t(s.m)), a)
    ctx.debug_set(nbm.NB_DBG_SYM_TILE, 5)
    assert torch.equal(ctx.accel(_t(s.x), _t(s.m)), a)
    comp = nbm.Context(G, eps, dt, precision="comp")
    assert comp.get_config(n)["threads"] == 64
    ac = comp.accel(_t(s.x, torch.float64), _t(s.m, torch.float64))
    assert rel_l2(to_np(ac), ref) <= 1e-6
    kdk = nbm.Context(G, eps, dt, scheme="kdk")
    x, v = _t(s.x), _t(s.v)
    kdk.run(x, v, _t(s.m), 3)
    xr, vr = oracle.run(s.x, s.v, s.m, G, eps, dt, 3, scheme="kdk")
    assert rel_l2(to_np(x), xr) <= 1e-5
    assert rel_l2(to_np(v), vr) <= 1e-4


def test_sym_accel_plummer_momentum(nbm):
    """Plummer sphere (the large-system workload's distribution): forces
    against the oracle, and the pair antisymmetry of the form itself: the
    mass-weighted sum of the forces is zero up to FP32 rounding of the sums."""
    n, G, eps = 20000, 1.0, 0.05
    s = ics.plummer(n, seed=5)
    ctx = _ctx(nbm, 1024, G, eps)
    a = to_np(ctx.accel(_t(s.x), _t(s.m)))
    assert rel_l2(a, oracle.accel(s.x, s.m, G, eps)) <= 2e-5
    p = (s.m[:, None] * a).sum(axis=0)
    scale = (s.m[:, None] * np.abs(a)).sum(axis=0)
    assert np.all(np.abs(p) <= 1e-5 * scale)


@pytest.mark.parametrize("scheme", ["paper", "kdk"])
@pytest.mark.parametrize("n,block", [(777, 512), (4096, 512), (3000, 256)])
def test_sym_run_matches_oracle(nbm, scheme, n, block):
    s = ics.cube(n, seed=40 + n)
    ctx = _ctx(nbm, block, G=1.0, eps=0.01, dt=1e-3, scheme=scheme)
    x, v, m = _t(s.x), _t(s.v), _t(s.m)
    before = ctx.launch_count
    ctx.run(x, v, m, 10)
    ctx.sync()
    # pack + (pair kernel + fixed-order sum) per step (+ the closing half kick)
    assert ctx.launch_count - before == 1 + 2 * (10 + (scheme == "kdk"))
    xr, vr = oracle.run(s.x, s.v, s.m, 1.0, 0.01, 1e-3, 10, scheme=scheme)
    assert rel_l2(to_np(x), xr) <= 1e-5
    assert rel_l2(to_np(v), vr) <= 1e-4


def test_sym_checkpoints_and_one_sided_agree(nbm):
    n, steps, k = 3000, 12, 4
    s = ics.cube(n, seed=9)
    out = {}
    for form in (1, 1024):
        ctx = _ctx(nbm, form)
        x, v, m = _t(s.x), _t(s.v), _t(s.m)
        ck = torch.zeros((steps // k + 1, n, 6), dtype=torch.float32, device=DEV)
        ctx.run(x, v, m, steps, ckpt=ck, ckpt_every=k)
        ctx.sync()
        out[form] = (to_np(x), to_np(v), to_np(ck))
    xs, vs, cs = out[1024]
    xo, vo, co = out[1]
    assert rel_l2(xs, xo) <= 1e-6 and rel_l2(vs, vo) <= 1e-5
    for slot in range(steps // k + 1):
        assert rel_l2(cs[slot], co[slot]) <= 1e-5
    assert np.array_equal(cs[-1][:, :3], xs) and np.array_equal(cs[-1][:, 3:], vs)


def test_sym_is_deterministic(nbm):
    n = 6000
    s = ics.plummer(n, seed=3)
    ctx = _ctx(nbm, 512, eps=0.05)
    a1 = ctx.accel(_t(s.x), _t(s.m)).clone()
    a2 = ctx.accel(_t(s.x), _t(s.m)).clone()
    ctx.sync()
    assert torch.equal(a1, a2)


def test_default_form_by_size(nbm):
    """Untuned forward, both precisions: one-sided below 16384 bodies,
    pair-symmetric from there, one-sided when pinned; the VJP (both
    precisions) from 8192."""
    ctx = nbm.Context(1.0, 0.01, 1e-3)
    if ctx.get_config(40000)["tuned"]:
        pytest.skip("a tuning table is loaded")
    assert ctx.get_config(12000)["form"] == "f32x2"
    assert ctx.get_config(20000)["form"] == "pair_symmetric"
    assert ctx.get_config(4000, nbm.MODE_ADJOINT)["form"] == "vjp"
    assert ctx.get_config(9000, nbm.MODE_ADJOINT)["form"] == "vjp_pair_symmetric"
    ctx.debug_set(nbm.NB_DBG_FORM, 1)
    assert ctx.get_config(40000)["form"] == "f32x2"
    comp = nbm.Context(1.0, 0.01, 1e-3, precision="comp")
    assert comp.get_config(12000)["form"] == "compensated"
    assert comp.get_config(20000)["form"] == "compensated_pair_symmetric"
    comp.debug_set(nbm.NB_DBG_FORM, 1)
    assert comp.get_config(40000)["form"] == "compensated"
    assert comp.get_config(4000, nbm.MODE_ADJOINT)["form"] == "vjp_compensated"
    assert comp.get_config(40000, nbm.MODE_ADJOINT)["form"] == "vjp_compensated_pair_symmetric"
    comp.debug_set(nbm.NB_DBG_VJP_FORM, 1)
    assert comp.get_config(40000, nbm.MODE_ADJOINT)["form"] == "vjp_compensated"


def test_sym_adjoint_matches_one_sided(nbm):
    """nb_adjoint recomputes each checkpoint segment with the forward force
    form: gradients with the pair-symmetric recompute agree with the
    one-sided ones."""
    n, T, k = 700, 12, 4
    s = ics.cube(n, seed=4)
    rng = np.random.default_rng(1)
    target = rng.uniform(-1, 1, (n, 3))
    grads = {}
    for form in (1, 512):
        ctx = _ctx(nbm, form)
        x0, v0, m = _t(s.x), _t(s.v), _t(s.m)
        ck = torch.zeros((T // k + 1, n, 6), dtype=torch.float32, device=DEV)
        x, v = x0.clone(), v0.clone()
        ctx.run(x, v, m, T, ckpt=ck, ckpt_every=k)
        xbar = 2 * (x - _t(target))
        vbar = torch.zeros_like(v)
        g = ctx.adjoint(m, T, ck, k, xbar, vbar)
        ctx.sync()
        grads[form] = [to_np(t) for t in g]
    for a, b in zip(grads[512], grads[1]):
        assert rel_l2(a, b) <= 1e-5


@pytest.mark.parametrize("form", [1, 512])
def test_step_buffer_padding_not_stale(nbm, form):
    """A context reused for a smaller system of the same padded size: the
    padding of the buffers that the steps write must not keep the larger
    system's bodies (they would act as extra masses from the second step)."""
    ctx = _ctx(nbm, form)
    big = ics.cube(1024, seed=11)
    x, v, m = _t(big.x), _t(big.v), _t(big.m * 50)
    ctx.run(x, v, m, 3)
    ctx.sync()
    n = 1000
    s = ics.cube(n, seed=12)
    x, v, m = _t(s.x), _t(s.v), _t(s.m)
    ctx.run(x, v, m, 6)
    ctx.sync()
    xr, vr = oracle.run(s.x, s.v, s.m, 1.0, 0.01, 1e-3, 6)
    assert rel_l2(to_np(x), xr) <= 1e-5
    assert rel_l2(to_np(v), vr) <= 1e-4


# ------------------------------------------------------------- adjoint VJP

@pytest.mark.parametrize("block", [256, 512])
@pytest.mark.parametrize("n", [2, 31, 64, 65, 257, 513, 2000])
def test_sym_vjp_matches_oracle(nbm, block, n):
    """The pair-symmetric VJP (each pair's x-bar and m-bar terms for both
    bodies from one evaluation; the own pair masked) against the FP64 oracle,
    at the one-sided FP32 VJP's tolerance."""
    G, eps = 1.0, 0.01
    s = ics.cube(n, seed=60 + n)
    ab = np.random.default_rng(n).normal(size=(n, 3))
    ctx = nbm.Context(G, eps, 1e-3)
    ctx.debug_set(nbm.NB_DBG_VJP_FORM, block)
    assert ctx.get_config(n, nbm.MODE_ADJOINT)["form"] == "vjp_pair_symmetric"
    xb, mb = ctx.vjp(_t(s.x), _t(s.m), _t(ab))
    rx, rm = oracle.vjp(s.x, s.m, G, eps, ab)
    assert rel_l2(to_np(xb), rx) <= 5e-5 and rel_l2(to_np(mb), rm) <= 5e-5


def test_sym_vjp_plummer_and_determinism(nbm):
    n, G, eps = 9000, 1.0, 0.05
    s = ics.plummer(n, seed=6)
    ab = np.random.default_rng(2).normal(size=(n, 3))
    ctx = nbm.Context(G, eps, 1e-3)
    ctx.debug_set(nbm.NB_DBG_VJP_FORM, 512)
    xb1, mb1 = ctx.vjp(_t(s.x), _t(s.m), _t(ab))
    xb2, mb2 = ctx.vjp(_t(s.x), _t(s.m), _t(ab))
    ctx.sync()
    assert torch.equal(xb1, xb2) and torch.equal(mb1, mb2)
    rx, rm = oracle.vjp(s.x, s.m, G, eps, ab)
    assert rel_l2(to_np(xb1), rx) <= 5e-5 and rel_l2(to_np(mb1), rm) <= 5e-5


@pytest.mark.parametrize("vjp_block", [256, 512])
def test_sym_adjoint_vs_fp64_oracle(nbm, vjp_block):
    """nb_adjoint with pair-symmetric forward recompute and VJP (N=64, T=20,
    the adjoint check size): the FP32 gradient against the FP64 oracle's,
    at the one-sided FP32 adjoint's bound."""
    n, T, k = 64, 20, 5
    s = ics.cube(n, seed=4, masses="equal")
    xstar = ics.targets(n, seed=4)
    G, eps, dt = 1.0, 0.01, 1e-3
    ctx = nbm.Context(G, eps, dt)
    ctx.debug_set(nbm.NB_DBG_FORM, 512)
    ctx.debug_set(nbm.NB_DBG_VJP_FORM, vjp_block)
    ctx.debug_set(nbm.NB_DBG_RUN_PATH, GRAPH)
    x, v, m = _t(s.x), _t(s.v), _t(s.m)
    ck = torch.empty((T // k + 1, n, 6), dtype=torch.float32, device=DEV)
    ctx.run(x, v, m, T, ckpt=ck, ckpt_every=k)
    xbT = 2 * (x - _t(xstar))
    got = ctx.adjoint(m, T, ck, k, xbT, torch.zeros_like(xbT))
    xT, _ = oracle.run(s.x, s.v, s.m, G, eps, dt, T)
    ref = oracle.adjoint(s.x, s.v, s.m, G, eps, dt, T, 2 * (xT - xstar), np.zeros((n, 3)))
    errs = [rel_l2(to_np(g), r) for g, r in zip(got, ref)]
    assert max(errs) <= 1e-3, errs


def test_sym_adjoint_midsize_matches_one_sided(nbm):
    """N = 3000, T = 24, k = 8: gradients with both pair-symmetric kernels
    against the all-one-sided run and the FP64 oracle."""
    n, T, k = 3000, 24, 8
    s = ics.cube(n, seed=14, masses="equal")
    xstar = ics.targets(n, seed=14)
    G, eps, dt = 1.0, 0.01, 1e-3
    grads = {}
    for form, vform in ((1, 1), (1024, 512)):
        ctx = nbm.Context(G, eps, dt)
        ctx.debug_set(nbm.NB_DBG_FORM, form)
        ctx.debug_set(nbm.NB_DBG_VJP_FORM, vform)
        ctx.debug_set(nbm.NB_DBG_RUN_PATH, GRAPH)
        x, v, m = _t(s.x), _t(s.v), _t(s.m)
        ck = torch.empty((T // k + 1, n, 6), dtype=torch.float32, device=DEV)
        ctx.run(x, v, m, T, ckpt=ck, ckpt_every=k)
        xbT = 2 * (x - _t(xstar))
        g = ctx.adjoint(m, T, ck, k, xbT, torch.zeros_like(xbT))
        ctx.sync()
        grads[form] = [to_np(t) for t in g]
    xT, _ = oracle.run(s.x, s.v, s.m, G, eps, dt, T)
    ref = oracle.adjoint(s.x, s.v, s.m, G, eps, dt, T, 2 * (xT - xstar), np.zeros((n, 3)))
    for a, b, r in zip(grads[1024], grads[1], ref):
        assert rel_l2(a, b) <= 1e-4
        assert rel_l2(a, r) <= 1e-3


# ----------------------------------------------------- precision form

@pytest.mark.parametrize("block", [256, 512, 1024])
@pytest.mark.parametrize("n", [2, 33, 1000, 4097, 20000])
def test_sym_compensated_accel_matches_oracle(nbm, block, n):
    """FP64 state, FP32 pair terms each evaluated once for both bodies, the
    block-pair partials two-summed: the precision form's 1e-6 bound."""
    G, eps = 1.0, 0.05
    s = ics.plummer(n, seed=40 + n)
    ctx = nbm.Context(G, eps, 5e-4, precision="comp")
    ctx.debug_set(nbm.NB_DBG_FORM, block)
    assert ctx.get_config(n)["form"] == "compensated_pair_symmetric"
    a = to_np(ctx.accel(_t(s.x, torch.float64), _t(s.m, torch.float64)))
    assert rel_l2(a, oracle.accel(s.x, s.m, G, eps)) <= 1e-6


@pytest.mark.parametrize("scheme", ["paper", "kdk"])
def test_sym_compensated_run_matches_oracle(nbm, scheme):
    n, G, eps, dt, T = 3000, 1.0, 0.05, 5e-4, 10
    s = ics.plummer(n, seed=2)
    ctx = nbm.Context(G, eps, dt, precision="comp", scheme=scheme)
    ctx.debug_set(nbm.NB_DBG_FORM, 512)
    ctx.debug_set(nbm.NB_DBG_RUN_PATH, GRAPH)
    f = torch.float64
    x, v, m = _t(s.x, f), _t(s.v, f), _t(s.m, f)
    ctx.run(x, v, m, T)
    xr, vr = oracle.run(s.x, s.v, s.m, G, eps, dt, T, scheme=scheme)
    assert rel_l2(to_np(x), xr) <= 1e-9
    assert rel_l2(to_np(v), vr) <= 1e-6


@pytest.mark.parametrize("block", [256, 512, 1024])
@pytest.mark.parametrize("n", [65536, 262144])
def test_sym_compensated_close_encounters(nbm, block, n):
    """The precision form's 1e-6 bound on close-encounter-heavy input: a
    uniform cube with eps = 0.01 (about 0.03 to 0.14 neighbours per body inside
    eps at these sizes), where each block-pair partial is an FP32 sum of up to
    the block's length of terms, some of them near the largest a pair can
    give (0.385 m / eps^2). Element-wise against the FP64 oracle on 1024
    sampled bodies, each block size pinned."""
    G, eps = 1.0, 0.01
    s = ics.cube(n, seed=17, masses="equal")
    ctx = nbm.Context(G, eps, 5e-4, precision="comp")
    ctx.debug_set(nbm.NB_DBG_FORM, block)
    assert ctx.get_config(n)["form"] == "compensated_pair_symmetric"
    a = to_np(ctx.accel(_t(s.x, torch.float64), _t(s.m, torch.float64)))
    idx = ics.subset_indices(n, 1024, 17 + block)
    err = rel_l2(a[idx], oracle.accel(s.x, s.m, G, eps, idx))
    print(f"precision form, cube eps=0.01, n={n}, block {block}: rel L2 {err:.3e}")
    assert err <= 1e-6


# ------------------------------------------------------------ tiled launches

@pytest.mark.parametrize("w", [1, 3, 7])
def test_sym_tiled_launches_bit_identical(nbm, w):
    """The pair-symmetric kernels launched tile by tile (w x w block pairs per
    launch, the partials of each tile folded into running sums in partner
    order) give bit for bit the results of one launch over all block pairs:
    forces, runs of both schemes (the precision form's with checkpoints), the
    precision form and the VJP, with ragged last strips (20 blocks of 1024
    bodies; 35 of 512 for the VJP)."""
    n = 20000
    s = ics.plummer(n, seed=31)
    G, eps = 1.0, 0.05
    ab = np.random.default_rng(5).normal(size=(n, 3))
    out = {}
    for tile in (-1, w):
        ctx = nbm.Context(G, eps, 1e-3)
        ctx.debug_set(nbm.NB_DBG_FORM, 1024)
        ctx.debug_set(nbm.NB_DBG_VJP_FORM, 512)
        ctx.debug_set(nbm.NB_DBG_RUN_PATH, GRAPH)
        ctx.debug_set(nbm.NB_DBG_SYM_TILE, tile)
        before = ctx.launch_count
        a = ctx.accel(_t(s.x), _t(s.m))
        ctx.sync()
        m_ = (20 + w - 1) // w
        # the pack, then one launch per tile and the final sum (or the pair kernel and its sum)
        assert ctx.launch_count - before == 1 + (m_ * (m_ + 1) // 2 + 1 if tile > 0 else 2)
        x, v, m = _t(s.x), _t(s.v), _t(s.m)
        ctx.run(x, v, m, 6)  # each position buffer read three times
        xb, mb = ctx.vjp(_t(s.x), _t(s.m), _t(ab))
        comp = nbm.Context(G, eps, 1e-3, precision="comp")
        comp.debug_set(nbm.NB_DBG_FORM, 1024)
        comp.debug_set(nbm.NB_DBG_SYM_TILE, tile)
        comp.debug_set(nbm.NB_DBG_RUN_PATH, GRAPH)
        ac = comp.accel(_t(s.x, torch.float64), _t(s.m, torch.float64))
        xc, vc = _t(s.x, torch.float64), _t(s.v, torch.float64)
        ck = torch.zeros((3, n, 6), dtype=torch.float64, device="cuda")
        comp.run(xc, vc, _t(s.m, torch.float64), 4, ckpt=ck, ckpt_every=2)
        kdk = nbm.Context(G, eps, 1e-3, scheme="kdk")
        kdk.debug_set(nbm.NB_DBG_FORM, 1024)
        kdk.debug_set(nbm.NB_DBG_RUN_PATH, GRAPH)
        kdk.debug_set(nbm.NB_DBG_SYM_TILE, tile)
        xk, vk = _t(s.x), _t(s.v)
        kdk.run(xk, vk, _t(s.m), 4)
        ctx.sync()
        comp.sync()
        kdk.sync()
        out[tile] = [t.clone() for t in (a, x, v, xb, mb, ac, xc, vc, ck, xk, vk)]
    for got, ref in zip(out[w], out[-1]):
        assert torch.equal(got, ref)
    assert rel_l2(to_np(out[w][0]), oracle.accel(s.x, s.m, G, eps)) <= 2e-5
    assert rel_l2(to_np(out[w][5]), oracle.accel(s.x, s.m, G, eps)) <= 1e-6


def test_sym_tiles_by_default_at_large_n(nbm):
    """Above 512 MiB of partials for one launch the forces go by tiles: at
    N = 262144 (1024-body blocks, 0.8 GB of partials in one launch) a step is
    the pack, one launch per tile and the final sum."""
    n = 262144
    ctx = nbm.Context(1.0, 0.05, 1e-3)
    if ctx.get_config(n)["tuned"]:
        pytest.skip("a tuning table is loaded")
    s = ics.plummer(n, seed=1)
    x, v, m = _t(s.x), _t(s.v), _t(s.m)
    before = ctx.launch_count
    ctx.run(x, v, m, 1)
    ctx.sync()
    assert ctx.launch_count - before > 3


def test_sym_two_million_bodies_sampled(nbm):
    """N = 2^21 Plummer in FP32: the pair-symmetric form (by tiles; one launch
    would need 51.5 GB of partials), 1024 sampled bodies against the FP64
    oracle at the plain FP32 bound."""
    n, G, eps = 1 << 21, 1.0, 0.05
    s = ics.plummer(n, seed=7)
    ctx = nbm.Context(G, eps, 1e-3)
    assert ctx.get_config(n)["form"] == "pair_symmetric"
    a = to_np(ctx.accel(_t(s.x), _t(s.m)))
    idx = ics.subset_indices(n, 1024, 8)
    err = rel_l2(a[idx], oracle.accel(s.x, s.m, G, eps, idx))
    print(f"N = 2^21 pair-symmetric (tiled) accel, 1024 sampled bodies: rel L2 {err:.3e}")
    assert err <= 2e-5


# ------------------------------------------- precision-form VJP, pair-symmetric

@pytest.mark.parametrize("block", [256, 512])
@pytest.mark.parametrize("n", [2, 65, 513, 2000, 9000])
def test_sym_vjp_compensated_matches_oracle(nbm, block, n):
    """The precision form's pair-symmetric VJP (FP64 state; d from the FP32
    (hi, lo) parts of the positions, FP32 sums within a block pair, the
    partials two-summed) against the FP64 oracle at the precision form's
    1e-6 bound, on a cube with eps = 0.01 (close pairs weigh as |d|^-5)."""
    G, eps = 1.0, 0.01
    s = ics.cube(n, seed=90 + n)
    ab = np.random.default_rng(n + 1).normal(size=(n, 3))
    ctx = nbm.Context(G, eps, 1e-3, precision="comp")
    ctx.debug_set(nbm.NB_DBG_VJP_FORM, block)
    assert ctx.get_config(n, nbm.MODE_ADJOINT)["form"] == "vjp_compensated_pair_symmetric"
    f = torch.float64
    xb, mb = ctx.vjp(_t(s.x, f), _t(s.m, f), _t(ab, f))
    rx, rm = oracle.vjp(s.x, s.m, G, eps, ab)
    ex, em = rel_l2(to_np(xb), rx), rel_l2(to_np(mb), rm)
    print(f"precision-form pair-symmetric VJP n={n} block {block}: xbar {ex:.2e}, mbar {em:.2e}")
    assert ex <= 1e-6 and em <= 1e-6


@pytest.mark.parametrize("vjp_block", [256, 512])
def test_sym_adjoint_precision_form_vs_fp64_oracle(nbm, vjp_block):
    """The precision-form adjoint (N = 64, T = 20, checkpoint every 5) with
    the pair-symmetric forward recompute and VJP against the FP64 oracle's
    gradient: within 1e-6 per block."""
    n, T, k = 64, 20, 5
    s = ics.cube(n, seed=4, masses="equal")
    xstar = ics.targets(n, seed=4)
    G, eps, dt = 1.0, 0.01, 1e-3
    f = torch.float64
    ctx = nbm.Context(G, eps, dt, precision="comp")
    ctx.debug_set(nbm.NB_DBG_FORM, 512)
    ctx.debug_set(nbm.NB_DBG_VJP_FORM, vjp_block)
    ctx.debug_set(nbm.NB_DBG_RUN_PATH, GRAPH)
    x, v, m = _t(s.x, f), _t(s.v, f), _t(s.m, f)
    ck = torch.empty((T // k + 1, n, 6), dtype=f, device=DEV)
    ctx.run(x, v, m, T, ckpt=ck, ckpt_every=k)
    xbT = 2 * (x - _t(xstar, f))
    got = ctx.adjoint(m, T, ck, k, xbT, torch.zeros_like(xbT))
    xT, _ = oracle.run(s.x, s.v, s.m, G, eps, dt, T)
    ref = oracle.adjoint(s.x, s.v, s.m, G, eps, dt, T, 2 * (xT - xstar), np.zeros((n, 3)))
    errs = [rel_l2(to_np(g), r) for g, r in zip(got, ref)]
    print("precision-form adjoint, pair-symmetric kernels: %s" % ["%.2e" % e for e in errs])
    assert max(errs) <= 1e-6, errs


def test_sym_tiled_adjoint_bit_identical(nbm):
    """nb_adjoint with the forward recompute and the VJP launched by tiles
    (the recompute on the adjoint's second stream with its own scratch)
    gives the gradients of one launch per kernel bit for bit, in both
    precisions."""
    n, T, k = 3000, 12, 4
    s = ics.cube(n, seed=23, masses="equal")
    xstar = ics.targets(n, seed=23)
    G, eps, dt = 1.0, 0.01, 1e-3
    for prec, f in (("fp32", torch.float32), ("comp", torch.float64)):
        grads = {}
        for tile in (-1, 2):
            ctx = nbm.Context(G, eps, dt, precision=prec)
            ctx.debug_set(nbm.NB_DBG_FORM, 512)
            ctx.debug_set(nbm.NB_DBG_VJP_FORM, 512)
            ctx.debug_set(nbm.NB_DBG_RUN_PATH, GRAPH)
            ctx.debug_set(nbm.NB_DBG_SYM_TILE, tile)
            x, v, m = _t(s.x, f), _t(s.v, f), _t(s.m, f)
            ck = torch.empty((T // k + 1, n, 6), dtype=f, device=DEV)
            ctx.run(x, v, m, T, ckpt=ck, ckpt_every=k)
            xbT = 2 * (x - _t(xstar, f))
            g = ctx.adjoint(m, T, ck, k, xbT, torch.zeros_like(xbT))
            ctx.sync()
            grads[tile] = [t.clone() for t in g]
        for a, b in zip(grads[2], grads[-1]):
            assert torch.equal(a, b), prec


def test_sym_adjoint_fused_preparation_bit_identical(nbm):
    """nb_adjoint with each reverse step prepared by the previous step's VJP
    epilogue (the default with a pair-symmetric VJP) gives the gradients of
    a preparation kernel per step bit for bit, in both precisions, by tiles
    and in one launch (the fused form's agreement with the FP64 oracle is
    the other adjoint tests', which run it by default)."""
    n, T, k = 3000, 12, 4
    s = ics.cube(n, seed=24, masses="equal")
    xstar = ics.targets(n, seed=24)
    G, eps, dt = 1.0, 0.01, 1e-3
    for prec, f in (("fp32", torch.float32), ("comp", torch.float64)):
        for tile in (-1, 3):
            grads = {}
            for prep in (1, 0):
                ctx = nbm.Context(G, eps, dt, precision=prec)
                ctx.debug_set(nbm.NB_DBG_VJP_FORM, 256)
                ctx.debug_set(nbm.NB_DBG_RUN_PATH, GRAPH)
                ctx.debug_set(nbm.NB_DBG_SYM_TILE, tile)
                ctx.debug_set(nbm.NB_DBG_ADJ_PREP, prep)
                x, v, m = _t(s.x, f), _t(s.v, f), _t(s.m, f)
                ck = torch.empty((T // k + 1, n, 6), dtype=f, device=DEV)
                ctx.run(x, v, m, T, ckpt=ck, ckpt_every=k)
                xbT = 2 * (x - _t(xstar, f))
                before = ctx.launch_count
                g = ctx.adjoint(m, T, ck, k, xbT, torch.zeros_like(xbT))
                ctx.sync()
                launches = ctx.launch_count - before
                grads[prep] = ([t.clone() for t in g], launches)
            for a, b in zip(grads[0][0], grads[1][0]):
                assert torch.equal(a, b), (prec, tile)
            # one preparation kernel per segment instead of one per step
            assert grads[1][1] - grads[0][1] == T - T // k
