"""Pins for the FP64 oracle against what the paper and the mathematics fix.

None of these checks re-types the oracle's own formula: each compares it with
an independent route (50-digit decimal brute force, a closed form, an
invariant, a symmetry, a convergence order, finite differences or an
independent autograd), chosen so that a dropped term, a flipped sign, a wrong
index or a transposed operand fails at least one of them.
"""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
from paper_2203_08263_gb300 import ics


# ---------------------------------------------------------------- brute force

def _dec_accel(x, m, G, eps):
    """Section 2.3 force sum in 50-digit decimal arithmetic, j = i included."""
    getcontext().prec = 50
    n = len(m)
    X = [[Decimal(float(c)) for c in row] for row in x]
    M = [Decimal(float(v)) for v in m]
    soft = Decimal(float(eps)) * Decimal(float(eps))
    out = []
    for i in range(n):
        acc = [Decimal(0)] * 3
        for j in range(n):
            d = [X[j][c] - X[i][c] for c in range(3)]
            s = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + soft
            w = M[j] / (s * s.sqrt())
            acc = [acc[c] + w * d[c] for c in range(3)]
        out.append([Decimal(float(G)) * a for a in acc])
    return out


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_accel_matches_decimal_brute_force(n):
    s = ics.cube(n, seed=100 + n)
    G, eps = 1.3, 0.05
    a = oracle.accel(s.x, s.m, G, eps)
    ref = np.array([[float(c) for c in row] for row in _dec_accel(s.x, s.m, G, eps)])
    if n == 1:
        assert np.all(a == 0.0)
        return
    assert _rel(a, ref) <= 1e-14


def test_step_matches_decimal_update():
    """One printed update (half kick, then drift with the new v) in decimal."""
    getcontext().prec = 50
    s = ics.cube(6, seed=7)
    G, eps, dt = 1.0, 0.01, 1e-3
    acc = _dec_accel(s.x, s.m, G, eps)
    DT = Decimal(dt)
    v_new = [[Decimal(float(s.v[i][c])) + acc[i][c] * DT / 2 for c in range(3)] for i in range(6)]
    x_new = [[Decimal(float(s.x[i][c])) + v_new[i][c] * DT for c in range(3)] for i in range(6)]
    x1, v1 = oracle.step(s.x, s.v, s.m, G, eps, dt)
    assert _rel(v1, [[float(c) for c in r] for r in v_new]) <= 1e-14
    assert _rel(x1, [[float(c) for c in r] for r in x_new]) <= 1e-14
    # the half kick and the new-v drift are what the paper prints; a full kick
    # or an old-v drift moves the result by O(dt^2 a), far above rounding
    a = oracle.accel(s.x, s.m, G, eps)
    full_kick_x = s.x + (s.v + a * dt) * dt
    old_v_x = s.x + s.v * dt
    assert _rel(x1, full_kick_x) > 1e-9
    assert _rel(x1, old_v_x) > 1e-9


def test_accel_subset_rows_equal_full_rows():
    """The i-subset branch of oracle.accel (the reference of every full-size
    GPU test) returns exactly the rows of the full sum: unsorted and repeated
    indices, both ends, a strided subset and the empty subset."""
    s = ics.plummer(700, seed=21)
    G, eps = 1.0, 0.05
    full = oracle.accel(s.x, s.m, G, eps)
    for idx in (np.array([0, 699, 350, 350, 1]), np.arange(700)[::-7], np.zeros(0, np.int64)):
        sub = oracle.accel(s.x, s.m, G, eps, idx)
        assert sub.shape == (len(idx), 3)
        assert np.array_equal(sub, full[idx])
    with pytest.raises(IndexError):
        oracle.accel(s.x, s.m, G, eps, np.array([700]))


def test_step_is_subset_accel_then_printed_update():
    """oracle.step on the rows of a subset is bit for bit the subset's
    oracle.accel followed by the printed half kick and drift with the new v
    (the composition that the full-size GPU step test uses as its
    reference)."""
    s = ics.cube(300, seed=22)
    G, eps, dt = 1.0, 0.01, 5e-4
    x1, v1 = oracle.step(s.x, s.v, s.m, G, eps, dt)
    idx = np.array([3, 0, 299, 150, 77])
    a = oracle.accel(s.x, s.m, G, eps, idx)
    v_ref = s.v[idx] + a * (dt / 2)
    x_ref = s.x[idx] + v_ref * dt
    assert np.array_equal(v1[idx], v_ref)
    assert np.array_equal(x1[idx], x_ref)


# ------------------------------------------------------------- closed forms

def test_two_body_closed_form_and_direction():
    G, eps = 2.0, 0.1
    x = np.array([[0.3, -0.2, 0.1], [1.1, 0.4, -0.5]])
    m = np.array([0.7, 1.9])
    a = oracle.accel(x, m, G, eps)
    d = x[1] - x[0]
    s = d @ d + eps * eps
    a0 = G * m[1] * d / s ** 1.5
    a1 = -G * m[0] * d / s ** 1.5
    assert np.allclose(a[0], a0, rtol=1e-15, atol=0)
    assert np.allclose(a[1], a1, rtol=1e-15, atol=0)
    # attraction: body 0 accelerates towards body 1
    assert a[0] @ d > 0 and a[1] @ d < 0


def test_zero_mass_body_feels_but_exerts_no_force():
    s = ics.cube(5, seed=3)
    m = s.m.copy()
    m[2] = 0.0
    G, eps = 1.0, 0.02
    a = oracle.accel(s.x, m, G, eps)
    keep = [0, 1, 3, 4]
    a_without = oracle.accel(s.x[keep], m[keep], G, eps)
    assert np.allclose(a[keep], a_without, rtol=1e-14, atol=0)
    assert np.linalg.norm(a[2]) > 0


def test_energy_closed_form_two_bodies():
    G, eps = 1.5, 0.2
    x = np.array([[0.0, 0.0, 0.0], [0.6, 0.8, 0.0]])
    v = np.array([[0.1, 0.2, 0.3], [-0.4, 0.5, 0.0]])
    m = np.array([2.0, 3.0])
    e = oracle.energy(x, v, m, G, eps)
    ke = 0.5 * 2.0 * (0.01 + 0.04 + 0.09) + 0.5 * 3.0 * (0.16 + 0.25)
    phi = -G * 6.0 / math.sqrt(1.0 + 0.04)
    assert e["KE"] == pytest.approx(ke, rel=1e-15)
    assert e["Phi"] == pytest.approx(phi, rel=1e-15)
    assert e["H"] == pytest.approx(ke + 0.5 * phi, rel=1e-15)
    assert np.allclose(e["P"], 2.0 * v[0] + 3.0 * v[1], rtol=1e-15)


# ----------------------------------------------------------------- invariants

def test_momentum_identity_and_step_momentum():
    s = ics.cube(200, seed=11)
    G, eps, dt = 1.0, 0.01, 1e-3
    a = oracle.accel(s.x, s.m, G, eps)
    ma = s.m[:, None] * a
    assert np.linalg.norm(ma.sum(axis=0)) <= 1e-14 * np.abs(ma).sum()
    x1, v1 = oracle.step(s.x, s.v, s.m, G, eps, dt)
    p0 = (s.m[:, None] * s.v).sum(axis=0)
    p1 = (s.m[:, None] * v1).sum(axis=0)
    assert np.linalg.norm(p1 - p0) <= 1e-15 * np.abs(s.m[:, None] * v1).sum()


def test_translation_rotation_scaling():
    s = ics.cube(30, seed=5)
    G, eps = 1.0, 0.03
    a = oracle.accel(s.x, s.m, G, eps)
    shift = np.array([3.0, -1.5, 0.25])
    assert _rel(oracle.accel(s.x + shift, s.m, G, eps), a) <= 1e-12
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1.0]])
    R = R @ np.array([[1, 0, 0], [0, math.cos(1.1), -math.sin(1.1)], [0, math.sin(1.1), math.cos(1.1)]])
    assert _rel(oracle.accel(s.x @ R.T, s.m, G, eps), a @ R.T) <= 1e-13
    lam = 2.5  # lengths and eps scaled together: a scales as lam^-2
    assert _rel(oracle.accel(lam * s.x, s.m, G, lam * eps), a / lam ** 2) <= 1e-13
    # permuting bodies permutes accelerations
    p = np.random.default_rng(0).permutation(30)
    assert _rel(oracle.accel(s.x[p], s.m[p], G, eps), a[p]) <= 1e-13


# ----------------------------------------------------- Kepler and convergence

def _kepler(G=1.0, eps=0.01, scheme="paper"):
    """Circular two-body orbit. Under the paper's update the single half kick
    per step makes the continuous dynamics Newtonian with G_eff = G/2; velocity
    Verlet (two half kicks) integrates full G."""
    m = np.array([0.5, 0.5])
    r = 1.0
    geff = G / 2.0 if scheme == "paper" else G
    omega = math.sqrt(geff * m.sum() / (r * r + eps * eps) ** 1.5)
    x0 = np.array([[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]])
    v0 = np.array([[0.0, 0.5 * omega, 0.0], [0.0, -0.5 * omega, 0.0]])
    return m, x0, v0, omega


def _kepler_err(dt, scheme, periods=1.0):
    G, eps = 1.0, 0.01
    m, x0, v0, omega = _kepler(G, eps, scheme)
    T = periods * 2 * math.pi / omega
    steps = int(round(T / dt))
    t = steps * dt
    x, _ = oracle.run(x0, v0, m, G, eps, dt, steps, scheme=scheme)
    exact = 0.5 * np.array([[math.cos(omega * t), math.sin(omega * t), 0.0]])
    exact = np.vstack([exact, -exact])
    return np.linalg.norm(x - exact) / np.linalg.norm(exact)


def test_kepler_circular_orbit_paper_update():
    assert _kepler_err(1e-4, "paper", periods=1.0) <= 2e-3
    # at half a period the O(dt) orbit-shape error of the half-kick/drift map
    # is at its largest (it closes again after a full period), so the order
    # shows cleanly there
    e1 = _kepler_err(1e-4, "paper", periods=0.5)
    e2 = _kepler_err(2e-4, "paper", periods=0.5)
    assert e1 <= 2e-3
    order = math.log2(e2 / e1)
    assert 0.9 <= order <= 1.1, order


def test_kepler_velocity_verlet_second_order():
    e1 = _kepler_err(1e-3, "kdk", periods=0.5)
    e2 = _kepler_err(2e-3, "kdk", periods=0.5)
    order = math.log2(e2 / e1)
    assert 1.8 <= order <= 2.2, order


def test_kepler_full_gravity_is_wrong_for_paper_update():
    """Under the printed update the orbit closes with G/2, not G: with G the
    same initial state is far from circular after one period."""
    G, eps = 1.0, 0.01
    m, x0, _, omega_half = _kepler(G, eps)
    omega_full = math.sqrt(G * m.sum() / (1 + eps * eps) ** 1.5)
    v0 = np.array([[0.0, 0.5 * omega_full, 0.0], [0.0, -0.5 * omega_full, 0.0]])
    dt = 1e-3
    steps = int(round(2 * math.pi / omega_full / dt))
    x, _ = oracle.run(x0, v0, m, G, eps, dt, steps)
    sep = np.linalg.norm(x[0] - x[1])
    assert abs(sep - 1.0) > 0.1


def _hprime_series(dt, periods, speed=0.8, chunks_per_period=50):
    """Relative deviation of H' = KE + Phi/2 sampled along a two-body orbit
    launched at `speed` times the circular speed (0.8: eccentric)."""
    G, eps = 1.0, 0.01
    m, x, v, omega = _kepler(G, eps)
    v = v * speed
    h0 = oracle.energy(x, v, m, G, eps)["H"]
    n = int(round(2 * math.pi / omega / dt / chunks_per_period))
    dev = []
    for _ in range(periods * chunks_per_period):
        x, v = oracle.run(x, v, m, G, eps, dt, n)
        dev.append(abs(oracle.energy(x, v, m, G, eps)["H"] - h0) / abs(h0))
    return np.array(dev)


def test_hprime_circular_orbit_drift():
    """10^4 steps at dt = 1e-4 on the circular orbit: |dH'|/|H'| <= 1e-6."""
    G, eps = 1.0, 0.01
    m, x, v, _ = _kepler(G, eps)
    h0 = oracle.energy(x, v, m, G, eps)["H"]
    x, v = oracle.run(x, v, m, G, eps, 1e-4, 10000)
    assert abs(oracle.energy(x, v, m, G, eps)["H"] - h0) <= 1e-6 * abs(h0)


def test_hprime_bounded_first_order_no_secular_drift():
    d1 = _hprime_series(1e-3, 4)
    d2 = _hprime_series(5e-4, 4)
    # the half-kick/drift map is symplectic Euler for H': the deviation of H'
    # is a bounded O(dt) oscillation
    assert d1.max() <= 1e-3
    assert 1.9 <= d1.max() / d2.max() <= 2.1
    # no secular growth: the last period is no worse than the first
    assert d1[-50:].max() <= 1.05 * d1[:50].max()


def test_hprime_conserved_many_bodies_small_dt():
    s = ics.cube(16, seed=21)
    G, eps = 1.0, 0.1
    h0 = oracle.energy(s.x, s.v, s.m, G, eps)["H"]
    e0 = oracle.energy(s.x, s.v, s.m, G, eps)
    x, v = oracle.run(s.x, s.v, s.m, G, eps, 1e-3, 2000)
    h1 = oracle.energy(x, v, s.m, G, eps)["H"]
    assert abs(h1 - h0) <= 2e-3 * abs(h0)
    # the physical E = KE + Phi is not what this update conserves
    e_phys0 = e0["KE"] + e0["Phi"]
    e1 = oracle.energy(x, v, s.m, G, eps)
    assert abs(e1["KE"] + e1["Phi"] - e_phys0) > 10 * abs(h1 - h0)
