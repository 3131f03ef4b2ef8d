"""Seeded synthetic initial conditions for the N-body workloads.

This module holds only input generation: random draws and the Plummer-sphere
sampling recipe. It contains none of the force or update arithmetic, so both
the CUDA path and the FP64 oracle may take their inputs from here.

The paper states its workload sizes (N = 256 ... 524288, 100 steps; Section
4.1) but not its initial conditions or constants: it defers the physics to an
external reference that is not available. The recipes below therefore stand
in for the paper's workloads:

* ``cube``: positions uniform in [-1, 1]^3, velocities uniform in
  [-0.1, 0.1]^3, masses either uniform in [0.5, 1.5]/N or equal to 1/N.
  Draw order from ``numpy.random.default_rng(seed)``: x (N, 3), then v (N, 3),
  then m (N) when masses are drawn.
* ``plummer``: the Aarseth, Henon & Wielen (1974) sampling of a Plummer
  sphere in units G = M = a = 1 with equal masses 1/N, radii truncated at 10,
  velocities from the isotropic distribution function by von Neumann
  rejection, then shifted to the centre-of-mass frame.
* ``ensemble``: 512 cube systems with sizes log-uniform in [64, 8192].
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = ["cube", "plummer", "ensemble", "targets", "System", "subset_indices"]


@dataclass
class System:
    x: np.ndarray  # (N, 3) float64
    v: np.ndarray  # (N, 3) float64
    m: np.ndarray  # (N,) float64

    @property
    def n(self) -> int:
        return int(self.m.shape[0])


def cube(n: int, seed: int, masses: str = "uniform", rng: np.random.Generator | None = None) -> System:
    """Uniform-cube system: x in [-1,1]^3, v in [-0.1,0.1]^3.

    ``masses="uniform"`` draws m uniform in [0.5, 1.5]/N after x and v;
    ``masses="equal"`` sets m = 1/N without a draw.
    """
    if rng is None:
        rng = np.random.default_rng(seed)
    x = rng.uniform(-1.0, 1.0, size=(n, 3))
    v = rng.uniform(-0.1, 0.1, size=(n, 3))
    if masses == "uniform":
        m = rng.uniform(0.5, 1.5, size=n) / n
    elif masses == "equal":
        m = np.full(n, 1.0 / n) if n > 0 else np.zeros(0)
    else:
        raise ValueError(f"unknown masses={masses!r}")
    return System(x, v, m)


def _isotropic(rng: np.random.Generator, radius: np.ndarray) -> np.ndarray:
    n = radius.shape[0]
    cos_t = rng.uniform(-1.0, 1.0, size=n)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    out = np.empty((n, 3))
    out[:, 0] = radius * sin_t * np.cos(phi)
    out[:, 1] = radius * sin_t * np.sin(phi)
    out[:, 2] = radius * cos_t
    return out


def plummer(n: int, seed: int, rmax: float = 10.0) -> System:
    """Plummer sphere, G = M = a = 1, equal masses 1/N (Aarseth et al. 1974).

    Radius from the cumulative mass fraction U: r = (U^(-2/3) - 1)^(-1/2),
    redrawn while r > rmax. Speed q * v_esc with v_esc = sqrt(2) (1+r^2)^(-1/4)
    and q drawn by rejection against g(q) = q^2 (1 - q^2)^(7/2) (whose maximum
    on [0, 1] is below 0.1). Directions isotropic. Finally the mass-weighted
    mean position and velocity are subtracted.
    """
    rng = np.random.default_rng(seed)
    r = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        u = rng.uniform(0.0, 1.0, size=todo.size)
        with np.errstate(divide="ignore", invalid="ignore"):
            rr = 1.0 / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        ok = np.isfinite(rr) & (rr <= rmax)
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    x = _isotropic(rng, r)
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        qq = rng.uniform(0.0, 1.0, size=todo.size)
        yy = rng.uniform(0.0, 0.1, size=todo.size)
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    vesc = math.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    v = _isotropic(rng, q * vesc)
    m = np.full(n, 1.0 / n)
    x -= (m[:, None] * x).sum(axis=0) / m.sum()
    v -= (m[:, None] * v).sum(axis=0) / m.sum()
    return System(x, v, m)


def ensemble_sizes(nsys: int, seed: int, nmin: int = 64, nmax: int = 8192,
                   rng: np.random.Generator | None = None) -> np.ndarray:
    """System sizes N = clamp(floor(exp(U(ln nmin, ln nmax))), nmin, nmax)."""
    if rng is None:
        rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(nmin), math.log(nmax), size=nsys)
    return np.clip(np.floor(np.exp(u)).astype(np.int64), nmin, nmax)


def ensemble(nsys: int = 512, seed: int = 3, nmin: int = 64, nmax: int = 8192):
    """Batched ensemble: sizes first, then each system's cube ICs in order.

    Returns (offsets[nsys+1] int64, x (sum N, 3), v (sum N, 3), m (sum N,)),
    every system with equal masses 1/N_s.
    """
    rng = np.random.default_rng(seed)
    sizes = ensemble_sizes(nsys, seed, nmin, nmax, rng=rng)
    offsets = np.zeros(nsys + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    xs, vs, ms = [], [], []
    for n in sizes:
        s = cube(int(n), seed, masses="equal", rng=rng)
        xs.append(s.x)
        vs.append(s.v)
        ms.append(s.m)
    return offsets, np.concatenate(xs), np.concatenate(vs), np.concatenate(ms)


def targets(n: int, seed: int, masses: str = "equal") -> np.ndarray:
    """Trajectory-loss targets x* uniform in [-1,1]^3, drawn after the system's
    own x, v (and m when drawn) from the same seeded stream."""
    rng = np.random.default_rng(seed)
    cube(n, seed, masses=masses, rng=rng)
    return rng.uniform(-1.0, 1.0, size=(n, 3))


def subset_indices(n: int, k: int, seed: int) -> np.ndarray:
    """First k entries of a seeded permutation of range(n), sorted."""
    perm = np.random.default_rng(seed).permutation(n)
    return np.sort(perm[:k]).astype(np.int64)
