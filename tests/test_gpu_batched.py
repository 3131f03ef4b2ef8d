"""GPU parity of the batched ensemble path (nb_run_batched): every system of
the batch against its own FP64 oracle run."""
import numpy as np
import pytest

import oracle
from paper_2203_08263_gb300 import ics
from gpu_util import ensure_built, rel_l2, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def nbm():
    ensure_built()
    from paper_2203_08263_gb300 import nbody
    return nbody


def _run(nbm, offsets, x, v, m, steps, eps=0.01, dt=1e-3, device_offsets=False):
    ctx = nbm.Context(1.0, eps, dt)
    xt = torch.tensor(x, dtype=torch.float32, device=DEV)
    vt = torch.tensor(v, dtype=torch.float32, device=DEV)
    mt = torch.tensor(m, dtype=torch.float32, device=DEV)
    off = torch.tensor(offsets, dtype=torch.int64)
    if device_offsets:
        off = off.to(DEV)
    ctx.run_batched(off, xt, vt, mt, steps)
    ctx.sync()
    return to_np(xt), to_np(vt), ctx


def test_small_ensemble_every_system(nbm):
    off, x, v, m = ics.ensemble(nsys=40, seed=11, nmin=64, nmax=1024)
    steps = 5
    gx, gv, _ = _run(nbm, off, x, v, m, steps)
    for s in range(40):
        a, b = off[s], off[s + 1]
        xr, vr = oracle.run(x[a:b], v[a:b], m[a:b], 1.0, 0.01, 1e-3, steps)
        assert rel_l2(gx[a:b], xr) <= 1e-5, s
        assert rel_l2(gv[a:b], vr) <= 1e-4, s


def test_ragged_and_empty_systems_device_offsets(nbm):
    sizes = [1, 0, 2, 3, 65, 130, 0, 257, 33]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (off[-1], 3))
    v = rng.uniform(-0.1, 0.1, (off[-1], 3))
    m = rng.uniform(0.5, 1.5, off[-1]) / 100
    gx, gv, _ = _run(nbm, off, x, v, m, 3, device_offsets=True)
    for s in range(len(sizes)):
        a, b = off[s], off[s + 1]
        if b == a:
            continue
        xr, _ = oracle.run(x[a:b], v[a:b], m[a:b], 1.0, 0.01, 1e-3, 3)
        assert rel_l2(gx[a:b], xr) <= 1e-5, s


def test_autotuned_batched_shape(nbm):
    off, x, v, m = ics.ensemble(nsys=60, seed=21, nmin=64, nmax=2048)
    ctx = nbm.Context(1.0, 0.01, 1e-3)
    offt = torch.tensor(off, dtype=torch.int64)
    assert not ctx.get_batched_config(offt)["tuned"]
    ctx.autotune_batched(offt)
    cfg = ctx.get_batched_config(offt)
    assert cfg["tuned"] and cfg["threads"] in (128, 256, 512)
    if cfg["form"] == "one_sided":
        assert cfg["bodies_per_thread"] in (1, 2, 4, 8) and cfg["jtile"] in (64, 128)
    else:
        assert (cfg["threads"], cfg["bodies_per_thread"], cfg["jtile"]) == (128, 8, 256)
    xt = torch.tensor(x, dtype=torch.float32, device=DEV)
    vt = torch.tensor(v, dtype=torch.float32, device=DEV)
    mt = torch.tensor(m, dtype=torch.float32, device=DEV)
    ctx.run_batched(offt, xt, vt, mt, 4)
    ctx.sync()
    for s in (0, 17, 59):
        a, b = off[s], off[s + 1]
        xr, _ = oracle.run(x[a:b], v[a:b], m[a:b], 1.0, 0.01, 1e-3, 4)
        assert rel_l2(to_np(xt)[a:b], xr) <= 1e-5


def test_c4_full_ensemble_sampled(nbm):
    """Batched ensemble: 512 cube systems, N log-uniform in [64, 8192]
    (seed 3), eps=0.01, dt=1e-3, 100 steps in one persistent launch, in both
    forms; the two largest and 30 seeded other systems against the oracle,
    positions and velocities."""
    off, x, v, m = ics.ensemble(nsys=512, seed=3)
    assert off[-1] > 800_000
    steps = 100
    sizes = np.diff(off)
    pick = list(np.argsort(sizes)[-2:]) + list(np.random.default_rng(3).choice(512, 30, replace=False))
    refs = {s: oracle.run(x[off[s]:off[s + 1]], v[off[s]:off[s + 1]], m[off[s]:off[s + 1]],
                          1.0, 0.01, 1e-3, steps) for s in pick}
    offt = torch.tensor(off, dtype=torch.int64)
    for form in ("one_sided", "pair_symmetric"):
        ctx = nbm.Context(1.0, 0.01, 1e-3)
        ctx.set_batched_form(offt, form)
        xt, vt, mt = (torch.tensor(a, dtype=torch.float32, device=DEV) for a in (x, v, m))
        ctx.run_batched(offt, xt, vt, mt, steps)
        ctx.sync()
        gx, gv = to_np(xt), to_np(vt)
        worst = 0.0
        for s in pick:
            a, b = off[s], off[s + 1]
            xr, vr = refs[s]
            ex, ev = rel_l2(gx[a:b], xr), rel_l2(gv[a:b], vr)
            worst = max(worst, ex)
            assert ex <= 1e-5 and ev <= 1e-4, (form, s, ex, ev)
        print(f"C4 {form}: worst x rel L2 over {len(pick)} systems {worst:.2e}")


# Sizes whose ragged rests need every item kind: rows of 128 i-bodies of
# 1..8 (in binary: 3 = 2 + 1, 7 = 4 + 2 + 1), a full chunk of 8 rows plus a rest, and tiny ones.
TAIL_SIZES = [1, 127, 128, 129, 300, 385, 640, 700, 896, 1000, 1024, 1025, 1500, 2047, 2200, 3]


@pytest.mark.parametrize("nt,r,jt", [(128, 1, 64), (128, 2, 128), (128, 4, 64), (128, 8, 64), (128, 8, 32),
                                     (256, 1, 64), (256, 4, 256), (256, 8, 128), (512, 1, 128),
                                     (512, 2, 64)])
def test_pinned_shapes_every_item_kind(nbm, nt, r, jt):
    sizes = TAIL_SIZES
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    rng = np.random.default_rng(100 + nt + r + jt)
    x = rng.uniform(-1, 1, (off[-1], 3))
    v = rng.uniform(-0.1, 0.1, (off[-1], 3))
    m = rng.uniform(0.5, 1.5, off[-1]) / 1000
    ctx = nbm.Context(1.0, 0.01, 1e-3)
    offt = torch.tensor(off, dtype=torch.int64)
    ctx.set_batched_config(offt, nt, r, jt)
    cfg = ctx.get_batched_config(offt)
    assert cfg["pinned"] and (cfg["threads"], cfg["bodies_per_thread"], cfg["jtile"]) == (nt, r, jt)
    xt = torch.tensor(x, dtype=torch.float32, device=DEV)
    vt = torch.tensor(v, dtype=torch.float32, device=DEV)
    mt = torch.tensor(m, dtype=torch.float32, device=DEV)
    ctx.run_batched(offt, xt, vt, mt, 3)
    ctx.sync()
    gx, gv = to_np(xt), to_np(vt)
    for s in range(len(sizes)):
        a, b = off[s], off[s + 1]
        xr, vr = oracle.run(x[a:b], v[a:b], m[a:b], 1.0, 0.01, 1e-3, 3)
        assert rel_l2(gx[a:b], xr) <= 1e-5, (s, sizes[s])
        assert rel_l2(gv[a:b], vr) <= 1e-4, (s, sizes[s])
    ctx.set_batched_config(offt, 0, 0, 0)
    assert not ctx.get_batched_config(offt)["pinned"]


def test_set_batched_config_rejects_bad_shapes(nbm):
    ctx = nbm.Context(1.0, 0.01, 1e-3)
    offt = torch.tensor([0, 100, 300], dtype=torch.int64)
    for nt, r, jt in ((128, 3, 64), (128, 16, 64), (128, 8, 48), (128, 8, 512), (128, 0, 64),
                      (512, 4, 64), (64, 1, 64), (0, 0, 64)):
        with pytest.raises(RuntimeError):
            ctx.set_batched_config(offt, nt, r, jt)


def test_batched_kdk_every_system(nbm):
    """Kick-drift-kick in the ensemble: each system against the oracle's KDK run."""
    off, x, v, m = ics.ensemble(nsys=24, seed=41, nmin=64, nmax=3000)
    ctx = nbm.Context(0.9, 0.02, 2e-3, scheme="kdk")
    xt = torch.tensor(x, dtype=torch.float32, device=DEV)
    vt = torch.tensor(v, dtype=torch.float32, device=DEV)
    mt = torch.tensor(m, dtype=torch.float32, device=DEV)
    ctx.run_batched(torch.tensor(off, dtype=torch.int64), xt, vt, mt, 6)
    ctx.sync()
    gx, gv = to_np(xt), to_np(vt)
    for s in range(24):
        a, b = off[s], off[s + 1]
        xr, vr = oracle.run(x[a:b], v[a:b], m[a:b], 0.9, 0.02, 2e-3, 6, scheme="kdk")
        assert rel_l2(gx[a:b], xr) <= 1e-5, s
        assert rel_l2(gv[a:b], vr) <= 1e-4, s


@pytest.mark.parametrize("scheme", ["paper", "kdk"])
def test_batched_precision_form_every_system(nbm, scheme):
    """FP64 state with compensated FP32 forces in the ensemble: every system at
    the tolerances of the single-system precision-form run (Plummer spheres)."""
    sizes = [3, 200, 1000, 1500, 2100, 700]
    parts = [ics.plummer(n, seed=60 + k) for k, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    x = np.concatenate([p.x for p in parts])
    v = np.concatenate([p.v for p in parts])
    m = np.concatenate([p.m for p in parts])
    ctx = nbm.Context(1.0, 0.05, 5e-4, precision="comp", scheme=scheme)
    xt = torch.tensor(x, dtype=torch.float64, device=DEV)
    vt = torch.tensor(v, dtype=torch.float64, device=DEV)
    mt = torch.tensor(m, dtype=torch.float64, device=DEV)
    offt = torch.tensor(off, dtype=torch.int64)
    cfg = ctx.get_batched_config(offt)
    assert cfg["form"] == "pair_symmetric" or cfg["bodies_per_thread"] <= 4
    ctx.run_batched(offt, xt, vt, mt, 10)
    ctx.sync()
    gx, gv = to_np(xt), to_np(vt)
    for s_ in range(len(sizes)):
        a, b = off[s_], off[s_ + 1]
        xr, vr = oracle.run(x[a:b], v[a:b], m[a:b], 1.0, 0.05, 5e-4, 10, scheme=scheme)
        assert rel_l2(gx[a:b], xr) <= 1e-9, s_
        assert rel_l2(gv[a:b], vr) <= 1e-6, s_


def test_batched_precision_form_tuned_and_pinned(nbm):
    off, x, v, m = ics.ensemble(nsys=30, seed=9, nmin=64, nmax=2048)
    ctx = nbm.Context(1.0, 0.01, 1e-3, precision="comp")
    offt = torch.tensor(off, dtype=torch.int64)
    with pytest.raises(RuntimeError):
        ctx.set_batched_config(offt, 256, 8, 64)  # above 4 bodies per thread
    ctx.autotune_batched(offt)
    cfg = ctx.get_batched_config(offt)
    assert cfg["tuned"] and (cfg["form"] == "pair_symmetric" or cfg["bodies_per_thread"] <= 4)
    xt = torch.tensor(x, dtype=torch.float64, device=DEV)
    vt = torch.tensor(v, dtype=torch.float64, device=DEV)
    mt = torch.tensor(m, dtype=torch.float64, device=DEV)
    ctx.run_batched(offt, xt, vt, mt, 4)
    ctx.sync()
    for s_ in (0, 11, 29):
        a, b = off[s_], off[s_ + 1]
        xr, _ = oracle.run(x[a:b], v[a:b], m[a:b], 1.0, 0.01, 1e-3, 4)
        assert rel_l2(to_np(xt)[a:b], xr) <= 1e-9


@pytest.mark.parametrize("form", ["one_sided", "pair_symmetric"])
def test_batched_padding_not_stale_after_other_plans(nbm, form):
    """Odd-sized systems read the padding half of their last pair record at
    every step. A context whose scratch last served other plans (a tuning run
    with another j-tile does exactly this) holds other bodies where this plan
    pads; the pack must clear the padding of both position buffers. The
    precision form's tolerances (1e-9 in x, 1e-6 in v after 4 steps) see one
    stale body of mass 1/N in a system."""
    sizes = [65, 129, 301, 777, 1023, 1]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    rng = np.random.default_rng(21)
    x = rng.uniform(-1, 1, (off[-1], 3))
    v = rng.uniform(-0.1, 0.1, (off[-1], 3))
    m = np.concatenate([np.full(n, 1.0 / n) for n in sizes])
    ctx = nbm.Context(1.0, 0.01, 1e-3, precision="comp")
    offt = torch.tensor(off, dtype=torch.int64)
    f = torch.float64
    # other plans first: two one-sided j-tiles and the other form, on shifted bodies
    for nt, r, jt in ((256, 1, 128), (128, 2, 64)):
        ctx.set_batched_config(offt, nt, r, jt)
        xs, vs, ms = (torch.tensor(a + 0.3, dtype=f, device=DEV) for a in (x, v, m))
        ctx.run_batched(offt, xs, vs, ms, 3)
    ctx.set_batched_config(offt, 0, 0, 0)
    ctx.set_batched_form(offt, "pair_symmetric" if form == "one_sided" else "one_sided")
    xs, vs, ms = (torch.tensor(a + 0.3, dtype=f, device=DEV) for a in (x, v, m))
    ctx.run_batched(offt, xs, vs, ms, 3)
    if form == "one_sided":
        ctx.set_batched_form(offt, None)
        ctx.set_batched_config(offt, 128, 4, 128)
    else:
        ctx.set_batched_form(offt, "pair_symmetric")
    assert ctx.get_batched_config(offt)["form"] == form
    xt, vt, mt = (torch.tensor(a, dtype=f, device=DEV) for a in (x, v, m))
    ctx.run_batched(offt, xt, vt, mt, 4)
    ctx.sync()
    gx, gv = to_np(xt), to_np(vt)
    for s_ in range(len(sizes)):
        a, b = off[s_], off[s_ + 1]
        xr, vr = oracle.run(x[a:b], v[a:b], m[a:b], 1.0, 0.01, 1e-3, 4)
        if sizes[s_] == 1:
            assert np.array_equal(gv[a:b], v[a:b])
            continue
        assert rel_l2(gx[a:b], xr) <= 1e-9, s_
        assert rel_l2(gv[a:b], vr) <= 1e-6, s_


# ------------------------------------------------- pair-symmetric form

SYM_SIZES = [1, 0, 2, 3, 65, 130, 0, 255, 256, 257, 33, 300, 513, 1000, 2047]


def _ens(sizes, seed, plummer=False):
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    if plummer:
        parts = [ics.plummer(n, seed=seed + k) for k, n in enumerate(sizes) if n > 0]
        x = np.concatenate([p.x for p in parts])
        v = np.concatenate([p.v for p in parts])
        m = np.concatenate([p.m for p in parts])
        return off, x, v, m
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, (off[-1], 3))
    v = rng.uniform(-0.1, 0.1, (off[-1], 3))
    m = rng.uniform(0.5, 1.5, off[-1]) / 1000
    return off, x, v, m


@pytest.mark.parametrize("scheme", ["paper", "kdk"])
def test_sym_ensemble_every_system(nbm, scheme):
    """The pair-symmetric ensemble form (groups of 256 bodies, one item per
    pair of groups and one epilogue item per group): every system of a batch
    with empty, tiny, exact-group and multi-group systems against its own
    oracle run."""
    off, x, v, m = _ens(SYM_SIZES, 7)
    ctx = nbm.Context(0.9, 0.02, 2e-3, scheme=scheme)
    offt = torch.tensor(off, dtype=torch.int64)
    ctx.set_batched_form(offt, "pair_symmetric")
    cfg = ctx.get_batched_config(offt)
    assert cfg["form"] == "pair_symmetric" and cfg["pinned"]
    xt = torch.tensor(x, dtype=torch.float32, device=DEV)
    vt = torch.tensor(v, dtype=torch.float32, device=DEV)
    mt = torch.tensor(m, dtype=torch.float32, device=DEV)
    ctx.run_batched(offt, xt, vt, mt, 6)
    ctx.sync()
    gx, gv = to_np(xt), to_np(vt)
    for s in range(len(SYM_SIZES)):
        a, b = off[s], off[s + 1]
        if b == a:
            continue
        xr, vr = oracle.run(x[a:b], v[a:b], m[a:b], 0.9, 0.02, 2e-3, 6, scheme=scheme)
        assert rel_l2(gx[a:b], xr) <= 1e-5, (s, SYM_SIZES[s])
        assert rel_l2(gv[a:b], vr) <= 1e-4, (s, SYM_SIZES[s])


def test_sym_ensemble_precision_form(nbm):
    sizes = [3, 200, 1000, 1500, 2100, 700]
    off, x, v, m = _ens(sizes, 60, plummer=True)
    ctx = nbm.Context(1.0, 0.05, 5e-4, precision="comp")
    offt = torch.tensor(off, dtype=torch.int64)
    ctx.set_batched_form(offt, "pair_symmetric")
    xt = torch.tensor(x, dtype=torch.float64, device=DEV)
    vt = torch.tensor(v, dtype=torch.float64, device=DEV)
    mt = torch.tensor(m, dtype=torch.float64, device=DEV)
    ctx.run_batched(offt, xt, vt, mt, 10)
    ctx.sync()
    gx, gv = to_np(xt), to_np(vt)
    for s_ in range(len(sizes)):
        a, b = off[s_], off[s_ + 1]
        xr, vr = oracle.run(x[a:b], v[a:b], m[a:b], 1.0, 0.05, 5e-4, 10)
        assert rel_l2(gx[a:b], xr) <= 1e-9, s_
        assert rel_l2(gv[a:b], vr) <= 1e-6, s_


def test_sym_ensemble_deterministic_and_agrees_with_one_sided(nbm):
    off, x, v, m = ics.ensemble(nsys=30, seed=5, nmin=64, nmax=3000)
    offt = torch.tensor(off, dtype=torch.int64)
    res = {}
    for form in ("pair_symmetric", "pair_symmetric", "one_sided"):
        ctx = nbm.Context(1.0, 0.01, 1e-3)
        ctx.set_batched_form(offt, form)
        xt = torch.tensor(x, dtype=torch.float32, device=DEV)
        vt = torch.tensor(v, dtype=torch.float32, device=DEV)
        mt = torch.tensor(m, dtype=torch.float32, device=DEV)
        ctx.run_batched(offt, xt, vt, mt, 5)
        ctx.sync()
        res.setdefault(form, []).append((to_np(xt), to_np(vt)))
    (x1, v1), (x2, v2) = res["pair_symmetric"]
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2)  # bit-identical repeats
    xo, vo = res["one_sided"][0]
    assert rel_l2(x1, xo) <= 1e-6 and rel_l2(v1, vo) <= 1e-5


def test_batched_form_default_and_pins(nbm):
    """Default form by the work estimate: pair-symmetric for the C4 size mix,
    one-sided for systems of 64 bodies; pins and their removal."""
    ctx = nbm.Context(1.0, 0.01, 1e-3)
    off, _, _, _ = ics.ensemble(nsys=512, seed=3)
    offt = torch.tensor(off, dtype=torch.int64)
    assert ctx.get_batched_config(offt)["form"] == "pair_symmetric"
    small = torch.tensor(np.arange(0, 64 * 41, 64), dtype=torch.int64)
    assert ctx.get_batched_config(small)["form"] == "one_sided"
    ctx.set_batched_form(small, "pair_symmetric")
    assert ctx.get_batched_config(small)["form"] == "pair_symmetric"
    ctx.set_batched_config(small, 256, 4, 64)  # a one-sided shape pins the one-sided form
    cfg = ctx.get_batched_config(small)
    assert cfg["form"] == "one_sided" and cfg["pinned"] and cfg["threads"] == 256
    ctx.set_batched_form(small, None)
    assert not ctx.get_batched_config(small)["pinned"]
    # one system of 2^20 bodies: its group-pair partials (48 GiB) exceed the cap
    big = torch.tensor([0, 1 << 20], dtype=torch.int64)
    assert ctx.get_batched_config(big)["form"] == "one_sided"
    with pytest.raises(nbm.NBodyError):
        ctx.set_batched_form(big, "pair_symmetric")


def test_sym_ensemble_wait_timeout_is_reported(nbm):
    """Pair-symmetric form with one warp holding back the release of its first
    item (a debug flag): the items that depend on it give up after 1 ms each,
    nb_sync reports NB_ERR_TIMEOUT, and the context then runs correctly."""
    sizes = [700, 300, 1000]
    off, x, v, m = _ens(sizes, 3)
    ctx = nbm.Context(1.0, 0.01, 1e-3)
    offt = torch.tensor(off, dtype=torch.int64)
    ctx.set_batched_form(offt, "pair_symmetric")

    def state():
        return (torch.tensor(x, dtype=torch.float32, device=DEV), torch.tensor(v, dtype=torch.float32, device=DEV),
                torch.tensor(m, dtype=torch.float32, device=DEV))

    ctx.debug_set(nbm.NB_DBG_WAIT_TIMEOUT_NS, 1_000_000)
    ctx.debug_set(nbm.NB_DBG_STALL_PRODUCER, 1)
    xt, vt, mt = state()
    ctx.run_batched(offt, xt, vt, mt, 3)
    with pytest.raises(nbm.NBodyError) as ei:
        ctx.sync()
    assert ei.value.status == nbm.NB_ERR_TIMEOUT
    ctx.debug_set(nbm.NB_DBG_STALL_PRODUCER, 0)
    ctx.debug_set(nbm.NB_DBG_WAIT_TIMEOUT_NS, 2_000_000_000)
    xt, vt, mt = state()
    ctx.run_batched(offt, xt, vt, mt, 3)
    ctx.sync()
    for s in range(len(sizes)):
        a, b = off[s], off[s + 1]
        xr, _ = oracle.run(x[a:b], v[a:b], m[a:b], 1.0, 0.01, 1e-3, 3)
        assert rel_l2(to_np(xt)[a:b], xr) <= 1e-5, s
