"""GPU parity of the forward path (nb_accel, nb_step, nb_run) against the FP64
oracle, through the C-ABI. Tolerances: accelerations relative L2 <= 2e-5 in
plain FP32, <= 1e-6 in the compensated precision form; positions after 10
steps <= 1e-4."""
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


def _t(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


SIZES = [1, 2, 3, 7, 8, 31, 32, 33, 255, 256, 257, 1000, 1024, 4097]


@pytest.mark.parametrize("n", SIZES)
def test_accel_fp32_matches_oracle(nbm, n):
    G, eps = 1.0, 0.01
    s = ics.cube(n, seed=1000 + n)
    ctx = nbm.Context(G, eps, 1e-3)
    a = to_np(ctx.accel(_t(s.x), _t(s.m)))
    ref = oracle.accel(s.x, s.m, G, eps)
    if n == 1:
        assert np.all(a == 0.0)
    else:
        assert rel_l2(a, ref) <= 2e-5


# every compiled shape, with forced multi-way j-splits and every j-tile size
SHAPES = [(128, 1, 0, 64), (128, 2, 3, 128), (128, 4, 0, 256), (128, 8, 5, 128),
          (256, 2, 2, 64), (256, 4, 7, 128), (256, 8, 1, 256)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("n", [33, 3001])
def test_accel_fp32_all_shapes(nbm, shape, n):
    G, eps = 0.7, 0.02
    s = ics.cube(n, seed=7 + n)
    ctx = nbm.Context(G, eps, 1e-3, tile_override=shape)
    a = to_np(ctx.accel(_t(s.x), _t(s.m)))
    assert rel_l2(a, oracle.accel(s.x, s.m, G, eps)) <= 2e-5


def test_autotuned_shape_matches_oracle(nbm):
    # the tuner times every compiled FP32 shape (packed and scalar) and keeps one
    n, G, eps = 2048, 1.0, 0.01
    s = ics.cube(n, seed=3)
    ctx = nbm.Context(G, eps, 1e-3)
    ctx.autotune(n)
    cfg = ctx.get_config(n)
    assert cfg["tuned"]
    a = to_np(ctx.accel(_t(s.x), _t(s.m)))
    assert rel_l2(a, oracle.accel(s.x, s.m, G, eps)) <= 2e-5


def test_accel_deterministic_and_host_path_identical(nbm):
    n, G, eps = 5000, 1.0, 0.01
    s = ics.cube(n, seed=5)
    ctx = nbm.Context(G, eps, 1e-3)
    x, m = _t(s.x), _t(s.m)
    a1 = ctx.accel(x, m).cpu()
    a2 = ctx.accel(x, m).cpu()
    assert torch.equal(a1, a2)
    xh = np.ascontiguousarray(s.x.astype(np.float32))
    mh = np.ascontiguousarray(s.m.astype(np.float32))
    ah = ctx.accel(xh, mh)
    assert np.array_equal(ah, a1.numpy())


def test_c1_positions_after_10_steps(nbm):
    """Plain method, small: N=1024 cube (seed 0), G=1, eps=0.01, dt=1e-3."""
    n, G, eps, dt, T = 1024, 1.0, 0.01, 1e-3, 10
    s = ics.cube(n, seed=0)
    ctx = nbm.Context(G, eps, dt)
    x, v, m = _t(s.x), _t(s.v), _t(s.m)
    ctx.run(x, v, m, T)
    ctx.sync()
    xr, vr = oracle.run(s.x, s.v, s.m, G, eps, dt, T)
    assert rel_l2(to_np(x), xr) <= 1e-4
    assert rel_l2(to_np(v), vr) <= 1e-4


def test_step_equals_run_and_host_run(nbm):
    n, G, eps, dt = 700, 1.0, 0.01, 1e-3
    s = ics.cube(n, seed=9)
    ctx = nbm.Context(G, eps, dt)
    x1, v1, m = _t(s.x), _t(s.v), _t(s.m)
    for _ in range(3):
        ctx.step(x1, v1, m)
    x2, v2 = _t(s.x), _t(s.v)
    ctx.run(x2, v2, m, 3)
    assert torch.equal(x1, x2) and torch.equal(v1, v2)
    xh = s.x.astype(np.float32).copy()
    vh = s.v.astype(np.float32).copy()
    ctx.run(xh, vh, s.m.astype(np.float32), 3)
    assert np.array_equal(xh, x1.cpu().numpy()) and np.array_equal(vh, v1.cpu().numpy())


def test_velocity_verlet_scheme(nbm):
    n, G, eps, dt, T = 512, 1.0, 0.01, 1e-3, 10
    s = ics.cube(n, seed=12)
    ctx = nbm.Context(G, eps, dt, scheme="kdk")
    x, v, m = _t(s.x), _t(s.v), _t(s.m)
    ctx.run(x, v, m, T)
    xr, vr = oracle.run(s.x, s.v, s.m, G, eps, dt, T, scheme="kdk")
    assert rel_l2(to_np(x), xr) <= 1e-4
    assert rel_l2(to_np(v), vr) <= 1e-4


def test_checkpoints_hold_the_trajectory(nbm):
    n, G, eps, dt, T, k = 300, 1.0, 0.01, 1e-3, 6, 2
    s = ics.cube(n, seed=13)
    ctx = nbm.Context(G, eps, dt)
    x, v, m = _t(s.x), _t(s.v), _t(s.m)
    ck = torch.empty((T // k + 1, n, 6), dtype=torch.float32, device=DEV)
    ctx.run(x, v, m, T, ckpt=ck, ckpt_every=k)
    ck = to_np(ck)
    assert np.array_equal(ck[0, :, :3], s.x.astype(np.float32))
    assert np.array_equal(ck[-1, :, :3], to_np(x))
    xr, vr = oracle.run(s.x, s.v, s.m, G, eps, dt, 2 * k)
    assert rel_l2(ck[2, :, :3], xr) <= 1e-5 and rel_l2(ck[2, :, 3:], vr) <= 1e-5


def test_zero_and_invalid(nbm):
    ctx = nbm.Context(1.0, 0.01, 1e-3)
    e = torch.empty((0, 3), device=DEV)
    ctx.run(e, e, torch.empty((0,), device=DEV), 5)
    with pytest.raises(nbm.NBodyError):
        ctx.run(_t(np.zeros((4, 3))), _t(np.zeros((4, 3))), _t(np.ones(4)), 4, ckpt=_t(np.zeros((3, 4, 6))),
                ckpt_every=3)
    with pytest.raises(nbm.NBodyError):
        nbm.Context(1.0, 0.0, 1e-3)


@pytest.mark.parametrize("what", ["accel", "run"])
def test_timeout_path_reports_and_context_recovers(nbm, what):
    """With the producer stalled no j-tile ever arrives: every bounded wait
    runs out after 1 ms, the call reports NB_ERR_TIMEOUT at nb_sync, and the
    context computes correctly afterwards."""
    n, G, eps = 4096, 1.0, 0.01
    s = ics.cube(n, seed=21)
    ctx = nbm.Context(G, eps, 1e-3)
    x, v, m = _t(s.x), _t(s.v), _t(s.m)
    ctx.debug_set(nbm.NB_DBG_WAIT_TIMEOUT_NS, 1_000_000)
    ctx.debug_set(nbm.NB_DBG_STALL_PRODUCER, 1)
    if what == "accel":
        ctx.accel(x, m)
    else:
        ctx.run(x.clone(), v.clone(), m, 2)
    with pytest.raises(nbm.NBodyError) as ei:
        ctx.sync()
    assert ei.value.status == nbm.NB_ERR_TIMEOUT
    ctx.sync()  # the error was reported once and cleared
    ctx.debug_set(nbm.NB_DBG_STALL_PRODUCER, 0)
    ctx.debug_set(nbm.NB_DBG_WAIT_TIMEOUT_NS, 2_000_000_000)
    a = to_np(ctx.accel(x, m))
    ctx.sync()
    assert rel_l2(a, oracle.accel(s.x, s.m, G, eps)) <= 2e-5


# ---------------------------------------------------------- precision form

@pytest.mark.parametrize("n", [2, 33, 1000, 4097])
def test_accel_compensated_matches_oracle(nbm, n):
    G, eps = 1.0, 0.05
    s = ics.plummer(n, seed=40 + n)
    ctx = nbm.Context(G, eps, 5e-4, precision="comp")
    a = to_np(ctx.accel(_t(s.x, torch.float64), _t(s.m, torch.float64)))
    assert rel_l2(a, oracle.accel(s.x, s.m, G, eps)) <= 1e-6


def test_c3_compensated_full_size_subset(nbm):
    """Precision form: N=1048576 Plummer (seed 2), eps=0.05; error on a
    4096-body random subset of i against the FP64 oracle."""
    n, G, eps = 1 << 20, 1.0, 0.05
    s = ics.plummer(n, seed=2)
    ctx = nbm.Context(G, eps, 5e-4, precision="comp")
    a = to_np(ctx.accel(_t(s.x, torch.float64), _t(s.m, torch.float64)))
    idx = ics.subset_indices(n, 4096, 2 + 1000)
    err = rel_l2(a[idx], oracle.accel(s.x, s.m, G, eps, idx))
    print(f"C3 compensated accel rel L2 on 4096-subset: {err:.3e}")
    assert err <= 1e-6


def test_c3_run_fp64_state(nbm):
    n, G, eps, dt, T = 2048, 1.0, 0.05, 5e-4, 10
    s = ics.plummer(n, seed=2)
    ctx = nbm.Context(G, eps, dt, precision="comp")
    x, v, m = _t(s.x, torch.float64), _t(s.v, torch.float64), _t(s.m, torch.float64)
    ctx.run(x, v, m, T)
    xr, vr = oracle.run(s.x, s.v, s.m, G, eps, dt, T)
    assert rel_l2(to_np(x), xr) <= 1e-9
    assert rel_l2(to_np(v), vr) <= 1e-6


def test_c3_full_size_step_subset(nbm):
    """Precision form at full size: one FP64-state step of N = 2^20 Plummer
    (seed 2, eps = 0.05, dt = 5e-4) through nb_step, in the form chosen for
    the size; the updated v and x of the 4096-body subset against the
    oracle's update of those bodies (its forces from all N bodies, then the
    printed half kick and drift; tests/test_oracle_pins.py pins this
    composition against oracle.step)."""
    n, G, eps, dt = 1 << 20, 1.0, 0.05, 5e-4
    s = ics.plummer(n, seed=2)
    ctx = nbm.Context(G, eps, dt, precision="comp")
    f = torch.float64
    x, v, m = _t(s.x, f), _t(s.v, f), _t(s.m, f)
    ctx.step(x, v, m)
    ctx.sync()
    idx = ics.subset_indices(n, 4096, 2 + 1000)
    a = oracle.accel(s.x, s.m, G, eps, idx)
    v_ref = s.v[idx] + a * (dt / 2)
    x_ref = s.x[idx] + v_ref * dt
    ev = rel_l2(to_np(v)[idx], v_ref)
    ex = rel_l2(to_np(x)[idx], x_ref)
    print(f"C3 one step, 4096 subset: v rel L2 {ev:.3e}, x rel L2 {ex:.3e}")
    assert ev <= 1e-6 and ex <= 1e-9


@pytest.mark.parametrize("form", [0, 1])
def test_c2_full_size_sampled(nbm, form):
    """Single large system: N=262144 Plummer (seed 1), eps=0.05, FP32;
    sampled outputs against the oracle, in the form chosen for the size (the
    pair-symmetric kernel untuned) and in the one-sided form."""
    n, G, eps = 262144, 1.0, 0.05
    s = ics.plummer(n, seed=1)
    ctx = nbm.Context(G, eps, 1e-3)
    ctx.debug_set(nbm.NB_DBG_FORM, form)
    a = to_np(ctx.accel(_t(s.x), _t(s.m)))
    idx = ics.subset_indices(n, 1024, 77)
    assert rel_l2(a[idx], oracle.accel(s.x, s.m, G, eps, idx)) <= 2e-5


# -------------------------------------------------------------- diagnostics

@pytest.mark.parametrize("prec", ["fp32", "comp"])
def test_energy_diagnostics(nbm, prec):
    n, G, eps = 3000, 1.0, 0.05
    s = ics.plummer(n, seed=8)
    dt_ = torch.float32 if prec == "fp32" else torch.float64
    ctx = nbm.Context(G, eps, 1e-3, precision=prec)
    x, v, m = _t(s.x, dt_), _t(s.v, dt_), _t(s.m, dt_)
    e = ctx.energy(x, v, m)
    xs, vs, ms = to_np(x), to_np(v), to_np(m)  # the state as stored
    r = oracle.energy(xs, vs, ms, G, eps)
    assert abs(e["KE"] - r["KE"]) <= 1e-12 * abs(r["KE"])
    assert np.allclose(e["P"], r["P"], rtol=0, atol=1e-12 * np.abs(ms[:, None] * vs).sum())
    assert abs(e["Phi"] - r["Phi"]) <= 1e-6 * abs(r["Phi"])
    # H' = KE + Phi/2 nearly cancels for a virialised sphere: bound it by the
    # size of its two terms
    assert abs(e["H"] - r["H"]) <= 1e-6 * (abs(r["KE"]) + 0.5 * abs(r["Phi"]))


@pytest.mark.parametrize("variant", [1, 2])
def test_denominator_ablation_variants_match_oracle(nbm, variant):
    """The sqrt-then-divide and powf denominators (the paper's math-operation
    experiment) compute the same forces."""
    n, G, eps = 3001, 1.0, 0.02
    s = ics.cube(n, seed=70 + variant)
    ctx = nbm.Context(G, eps, 1e-3)
    ctx.debug_set(nbm.NB_DBG_MATH_VARIANT, variant)
    a = to_np(ctx.accel(_t(s.x), _t(s.m)))
    assert rel_l2(a, oracle.accel(s.x, s.m, G, eps)) <= 2e-5
    x, v, m = _t(s.x), _t(s.v), _t(s.m)
    ctx.run(x, v, m, 3)
    xr, _ = oracle.run(s.x, s.v, s.m, G, eps, 1e-3, 3)
    assert rel_l2(to_np(x), xr) <= 1e-5


def test_measured_peaks_are_physical(nbm):
    ctx = nbm.Context(1.0, 0.01, 1e-3)
    p = ctx.measure_peaks()
    nominal = torch.cuda.get_device_properties(0).multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    # a plain FMA stream cannot beat the FMA lanes at the maximum clock
    assert 0.5 * nominal < p["ffma_tflops"] <= 1.02 * nominal
    assert 0.5 * nominal < p["ffma2_tflops"] <= 1.02 * nominal
    assert p["mufu_rsqrt_gops"] > 0


def test_misaligned_and_foreign_pointers_rejected(nbm):
    ctx = nbm.Context(1.0, 0.01, 1e-3)
    x = torch.zeros(3 * 64 + 1, device=DEV)
    m = torch.ones(64, device=DEV)
    lib = nbm.load()
    a = torch.empty((64, 3), device=DEV)
    stream = torch.cuda.current_stream().cuda_stream
    # a float32 array that starts 2 bytes into an allocation
    st = lib.nb_accel(ctx.h, 64, x.data_ptr() + 2, m.data_ptr(), a.data_ptr(), stream)
    assert st == nbm.NB_ERR_INVALID
    assert b"aligned" in lib.nb_last_error(ctx.h)
    st = lib.nb_accel(ctx.h, 64, None, m.data_ptr(), a.data_ptr(), stream)
    assert st == nbm.NB_ERR_INVALID
    assert lib.nb_run(ctx.h, -1, x.data_ptr(), x.data_ptr(), m.data_ptr(), 1, None, 0, stream) == nbm.NB_ERR_INVALID
    assert lib.nb_run(ctx.h, 64, x.data_ptr(), x.data_ptr(), m.data_ptr(), -3, None, 0, stream) == nbm.NB_ERR_INVALID
