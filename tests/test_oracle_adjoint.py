"""Pins for the oracle's reverse mode (vector-Jacobian product and trajectory
adjoint): finite differences of the forward oracle, an independent PyTorch
FP64 autograd of the plain force formula, and the dot-product identity."""
import numpy as np
import pytest

import oracle
from paper_2203_08263_gb300 import ics

torch = pytest.importorskip("torch")


def _torch_accel(x, m, G, eps):
    """Plain broadcast form of the Section 2.3 force sum (CPU, float64)."""
    d = x[None, :, :] - x[:, None, :]          # d[i, j] = x_j - x_i
    s = (d * d).sum(-1) + eps * eps
    return G * (m[None, :, None] * d * s[:, :, None] ** -1.5).sum(1)


def test_vjp_matches_torch_autograd():
    s = ics.cube(40, seed=31)
    G, eps = 1.2, 0.02
    abar = np.random.default_rng(1).normal(size=(40, 3))
    xb, mb = oracle.vjp(s.x, s.m, G, eps, abar)
    xt = torch.tensor(s.x, dtype=torch.float64, requires_grad=True)
    mt = torch.tensor(s.m, dtype=torch.float64, requires_grad=True)
    a = _torch_accel(xt, mt, G, eps)
    gx, gm = torch.autograd.grad(a, (xt, mt), torch.tensor(abar))
    assert np.linalg.norm(xb - gx.numpy()) <= 1e-12 * np.linalg.norm(gx.numpy())
    assert np.linalg.norm(mb - gm.numpy()) <= 1e-12 * np.linalg.norm(gm.numpy())


def test_vjp_dot_product_identity_against_fd_jvp():
    """<J dx, abar> = <dx, J^T abar>, with J dx from central differences of
    the forward oracle (no derivative code involved)."""
    s = ics.cube(24, seed=9)
    G, eps = 1.0, 0.05
    rng = np.random.default_rng(2)
    abar = rng.normal(size=(24, 3))
    dx = rng.normal(size=(24, 3))
    dm = rng.normal(size=24) * s.m
    h = 1e-6
    jdx = (oracle.accel(s.x + h * dx, s.m, G, eps) - oracle.accel(s.x - h * dx, s.m, G, eps)) / (2 * h)
    jdm = (oracle.accel(s.x, s.m + h * dm, G, eps) - oracle.accel(s.x, s.m - h * dm, G, eps)) / (2 * h)
    xb, mb = oracle.vjp(s.x, s.m, G, eps, abar)
    lhs = (jdx * abar).sum()
    assert lhs == pytest.approx((dx * xb).sum(), rel=1e-7)
    assert (jdm * abar).sum() == pytest.approx((dm * mb).sum(), rel=1e-7)


def _loss(x0, v0, m, G, eps, dt, T, xstar):
    xT, _ = oracle.run(x0, v0, m, G, eps, dt, T)
    return float(((xT - xstar) ** 2).sum())


def test_adjoint_matches_central_differences_n64_t20():
    """The trajectory-loss gradient w.r.t. x0, v0 and m against central
    differences, h = 1e-6 max(1, |theta|), relative L2 <= 1e-4 per block."""
    n, T, G, eps, dt = 64, 20, 1.0, 0.01, 1e-3
    s = ics.cube(n, seed=4, masses="equal")
    xstar = ics.targets(n, seed=4)
    xT, vT = oracle.run(s.x, s.v, s.m, G, eps, dt, T)
    gx, gv, gm = oracle.adjoint(s.x, s.v, s.m, G, eps, dt, T, 2 * (xT - xstar), np.zeros((n, 3)))

    def fd(which):
        base = {"x": s.x, "v": s.v, "m": s.m}[which]
        out = np.zeros_like(base)
        flat = out.reshape(-1)
        for k in range(base.size):
            th = base.reshape(-1)[k]
            h = 1e-6 * max(1.0, abs(th))
            args = []
            for sgn in (1.0, -1.0):
                p = base.copy().reshape(-1)
                p[k] = th + sgn * h
                p = p.reshape(base.shape)
                kw = {"x": s.x, "v": s.v, "m": s.m}
                kw[which] = p
                args.append(_loss(kw["x"], kw["v"], kw["m"], G, eps, dt, T, xstar))
            flat[k] = (args[0] - args[1]) / (2 * h)
        return out

    for got, which in ((gx, "x"), (gv, "v"), (gm, "m")):
        ref = fd(which)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-4, (which, err)


def test_adjoint_matches_torch_autograd_through_trajectory():
    n, T, G, eps, dt = 16, 12, 1.0, 0.05, 2e-3
    s = ics.cube(n, seed=17)
    xstar = ics.targets(n, seed=17, masses="uniform")
    x = torch.tensor(s.x, requires_grad=True)
    v = torch.tensor(s.v, requires_grad=True)
    m = torch.tensor(s.m, requires_grad=True)
    xs, vs = x, v
    for _ in range(T):
        vs = vs + _torch_accel(xs, m, G, eps) * dt / 2.0
        xs = xs + vs * dt
    loss = ((xs - torch.tensor(xstar)) ** 2).sum() + (vs ** 2).sum()
    gx, gv, gm = torch.autograd.grad(loss, (x, v, m))
    xT, vT = oracle.run(s.x, s.v, s.m, G, eps, dt, T)
    ox, ov, om = oracle.adjoint(s.x, s.v, s.m, G, eps, dt, T, 2 * (xT - xstar), 2 * vT)
    for a, b in ((ox, gx), (ov, gv), (om, gm)):
        b = b.numpy()
        assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(b)
