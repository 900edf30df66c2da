"""Seeded synthetic inputs shaped like the NURBS-Diff fitting workloads.

This module holds no NURBS arithmetic: it only draws knot vectors, control nets,
weights and parameter grids with numpy's ``default_rng``.  It is the one module
shared by the CUDA path's tests and benchmark and by the CPU oracle's tests.

Shapes and distributions follow the paper's workloads:

* surfaces: bicubic, control nets of 6..64 per direction, 64^2..512^2 sample
  grids (Sec. 5.3 and the test-surface table of the appendix);
* curves: cubic, 16..64 control points, uniformly spaced samples (Sec. 5.1).

Sample grids are uniform on [0, 1] inclusive of both ends (u_a = a / (N-1)),
computed in float64 and rounded once to float32; the same float32 values feed
every implementation.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def uniform_params(count: int) -> np.ndarray:
    """u_a = a / (count-1) for a < count, rounded once to float32 (count == 1 -> [0])."""
    if count <= 1:
        return np.zeros(max(count, 0), dtype=np.float32)
    return (np.arange(count, dtype=np.float64) / (count - 1)).astype(np.float32)


def clamped_uniform_knots(n1: int, p: int) -> np.ndarray:
    """0^(p+1), k/(n1-p) for k = 1..n1-p-1, 1^(p+1); float32."""
    interior = np.arange(1, n1 - p, dtype=np.float64) / (n1 - p)
    return np.concatenate([np.zeros(p + 1), interior, np.ones(p + 1)]).astype(np.float32)


def clamped_random_knots(rng: np.random.Generator, n1: int, p: int, min_gap: float = 1e-3) -> np.ndarray:
    """Clamped knot vector with n1-p-1 sorted U[0,1] interior knots, redrawn until
    every gap (including the gaps to 0 and to 1) is at least ``min_gap`` after
    rounding to float32."""
    k = n1 - p - 1
    while True:
        inner = np.sort(rng.uniform(0.0, 1.0, size=k)).astype(np.float32)
        full = np.concatenate([[0.0], inner.astype(np.float64), [1.0]])
        if k == 0 or np.min(np.diff(full)) >= min_gap:
            break
    return np.concatenate([np.zeros(p + 1, np.float32), inner, np.ones(p + 1, np.float32)]).astype(np.float32)


def planar_net(rng: np.random.Generator, n1: int, m1: int, z_sigma: float = 0.05,
               w_lo: float = 0.5, w_hi: float = 2.0) -> np.ndarray:
    """[n1, m1, 4] float32: x = i/(n1-1), y = j/(m1-1), z ~ N(0, z_sigma), w ~ U[w_lo, w_hi]."""
    x = np.linspace(0.0, 1.0, n1)[:, None] * np.ones((1, m1))
    y = np.ones((n1, 1)) * np.linspace(0.0, 1.0, m1)[None, :]
    z = rng.normal(0.0, z_sigma, size=(n1, m1))
    w = rng.uniform(w_lo, w_hi, size=(n1, m1))
    return np.stack([x, y, z, w], axis=-1).astype(np.float32)


def random_walk_polygon(rng: np.random.Generator, n1: int, step: float = 0.1,
                        w_lo: float = 0.5, w_hi: float = 2.0) -> np.ndarray:
    """[n1, 4] float32: a 3-D random walk from the origin with N(0, step) steps, w ~ U[w_lo, w_hi]."""
    steps = rng.normal(0.0, step, size=(n1, 3))
    steps[0] = 0.0
    pts = np.cumsum(steps, axis=0)
    w = rng.uniform(w_lo, w_hi, size=(n1, 1))
    return np.concatenate([pts, w], axis=1).astype(np.float32)


@dataclass
class Surface:
    """One NURBS surface: degrees, knots, control net [n1, m1, 4] and sample grids."""
    p: int
    q: int
    U: np.ndarray
    V: np.ndarray
    ctrl: np.ndarray
    u: np.ndarray
    v: np.ndarray

    @property
    def n1(self) -> int:
        return self.ctrl.shape[0]

    @property
    def m1(self) -> int:
        return self.ctrl.shape[1]

    @property
    def npts(self) -> int:
        return len(self.u) * len(self.v)


@dataclass
class Curve:
    """One NURBS curve: degree, knots, control polygon [n1, 4] and samples."""
    p: int
    U: np.ndarray
    ctrl: np.ndarray
    u: np.ndarray

    @property
    def n1(self) -> int:
        return self.ctrl.shape[0]

    @property
    def npts(self) -> int:
        return len(self.u)


def surface(rng, p=3, q=3, n1=16, m1=16, nu=64, nv=64, knots="random", min_gap=1e-3,
            z_sigma=0.05) -> Surface:
    if knots == "uniform":
        U, V = clamped_uniform_knots(n1, p), clamped_uniform_knots(m1, q)
    else:
        U, V = clamped_random_knots(rng, n1, p, min_gap), clamped_random_knots(rng, m1, q, min_gap)
    ctrl = planar_net(rng, n1, m1, z_sigma)
    return Surface(p, q, U, V, ctrl, uniform_params(nu), uniform_params(nv))


def twin_net(rng, s: Surface) -> Surface:
    """A surface with the same degrees, knots and grid as ``s`` and an independently
    drawn control net (the fitting target of the batched fit workloads)."""
    return Surface(s.p, s.q, s.U, s.V, planar_net(rng, s.n1, s.m1), s.u, s.v)


def curve(rng, p=3, n1=64, nu=1024, knots="random", min_gap=1e-3) -> Curve:
    U = clamped_uniform_knots(n1, p) if knots == "uniform" else clamped_random_knots(rng, n1, p, min_gap)
    return Curve(p, U, random_walk_polygon(rng, n1), uniform_params(nu))


def twin_polygon(rng, c: Curve) -> Curve:
    return Curve(c.p, c.U, random_walk_polygon(rng, c.n1), c.u)


# ------------------------------------------------------------ workload shapes
def single_bicubic(seed: int = 0) -> Surface:
    """One bicubic surface, 16x16 net, clamped uniform knots, 64x64 grid."""
    return surface(np.random.default_rng(seed), 3, 3, 16, 16, 64, 64, knots="uniform")


def bicubic_batch(seed: int = 0, batch: int = 256, net: int = 32, grid: int = 128):
    """``batch`` bicubic surfaces with net x net control nets, random clamped knots
    (min gap 1e-3) and grid x grid samples, plus an independent target net each."""
    rng = np.random.default_rng(seed)
    rng_t = np.random.default_rng(seed + 1)
    surfs = [surface(rng, 3, 3, net, net, grid, grid) for _ in range(batch)]
    targets = [twin_net(rng_t, s) for s in surfs]
    return surfs, targets


def cubic_curve_batch(seed: int = 0, batch: int = 4096, n1: int = 64, samples: int = 1024):
    rng = np.random.default_rng(seed)
    rng_t = np.random.default_rng(seed + 1)
    curves = [curve(rng, 3, n1, samples) for _ in range(batch)]
    targets = [twin_polygon(rng_t, c) for c in curves]
    return curves, targets


def ragged_batch(seed: int = 0, batch: int = 1000, deg=(2, 5), net=(8, 64), grid=(32, 256)):
    """Uneven batch: degrees, net sizes and grid sizes drawn uniformly per direction
    (net >= degree + 1), random clamped knots, plus an independent target net each."""
    rng = np.random.default_rng(seed)
    rng_t = np.random.default_rng(seed + 1)
    surfs = []
    for _ in range(batch):
        p, q = (int(x) for x in rng.integers(deg[0], deg[1] + 1, size=2))
        n1 = int(rng.integers(max(net[0], p + 1), net[1] + 1))
        m1 = int(rng.integers(max(net[0], q + 1), net[1] + 1))
        nu, nv = (int(x) for x in rng.integers(grid[0], grid[1] + 1, size=2))
        surfs.append(surface(rng, p, q, n1, m1, nu, nv))
    targets = [twin_net(rng_t, s) for s in surfs]
    return surfs, targets

def double_curved_net(n1: int = 12, amp: float = 0.25, rng: np.random.Generator | None = None,
                      w_lo: float = 1.0, w_hi: float = 1.0) -> np.ndarray:
    """A double-curved patch: z = amp sin(pi x) cos(pi y) sampled on an n1 x n1
    grid of control points over [0,1]^2; weights U[w_lo, w_hi] (1 by default)."""
    g = np.linspace(0.0, 1.0, n1, dtype=np.float64)
    X, Y = np.meshgrid(g, g, indexing="ij")
    net = np.zeros((n1, n1, 4), np.float32)
    net[..., 0], net[..., 1] = X, Y
    net[..., 2] = amp * np.sin(np.pi * X) * np.cos(np.pi * Y)
    net[..., 3] = 1.0 if rng is None else rng.uniform(w_lo, w_hi, size=(n1, n1))
    return net


def offset_batch(seed: int = 0, batch: int = 4096, n1: int = 12, grid: int = 20):
    """Bicubic double-curved patches (random amplitude and weights U[0.8, 1.2],
    uniform knots) sampled on grid x grid points: the shape of the paper's
    offsetting test surfaces."""
    rng = np.random.default_rng(seed)
    U = clamped_uniform_knots(n1, 3)
    out = []
    for _ in range(batch):
        net = double_curved_net(n1, float(rng.uniform(0.1, 0.3)), rng, 0.8, 1.2)
        out.append(Surface(3, 3, U, U, net, uniform_params(grid), uniform_params(grid)))
    return out
