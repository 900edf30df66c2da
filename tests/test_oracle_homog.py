"""Pins of the oracle's gradient with respect to the homogeneous control points
Pw = (w x, w y, w z, w) (Eq. 3 written homogeneously): central finite differences
taken in the homogeneous coordinates, through the Cartesian forward."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_14547_gb300 import synth


def _cart(pw):
    c = pw.copy()
    c[..., :3] = pw[..., :3] / pw[..., 3:4]
    return c


def _homog(ctrl):
    pw = ctrl.copy()
    pw[..., :3] = ctrl[..., :3] * ctrl[..., 3:4]
    return pw


def _fd(L, pw, grad, h=1e-6, rtol=1e-6):
    flat = pw.reshape(-1)
    for idx in range(flat.size):
        xp, xm = flat.copy(), flat.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (L(xp.reshape(pw.shape)) - L(xm.reshape(pw.shape))) / (2 * h)
        g = grad.reshape(-1)[idx]
        assert abs(fd - g) <= rtol * max(abs(fd), abs(g), 1e-3), (idx, fd, g)


@pytest.mark.parametrize("seed,p,q", [(0, 3, 2), (1, 1, 4), (2, 2, 2)])
def test_surface_homogeneous_gradient_central_differences(seed, p, q):
    rng = np.random.default_rng(seed)
    s = synth.surface(rng, p, q, 6, 6, 7, 6, knots="random", min_gap=0.02)
    ctrl = s.ctrl.astype(np.float64)
    ctrl[..., :3] += rng.normal(0, 0.3, size=ctrl[..., :3].shape)
    g = rng.normal(size=(len(s.u), len(s.v), 3))

    def L(pw):
        return float((O.surface_eval(p, q, s.U, s.V, _cart(pw), s.u, s.v) * g).sum())

    dpw = O.surface_vjp_homog(p, q, s.U, s.V, ctrl, s.u, s.v, g)
    _fd(L, _homog(ctrl), dpw)


@pytest.mark.parametrize("seed,p", [(3, 3), (4, 1), (5, 5)])
def test_curve_homogeneous_gradient_central_differences(seed, p):
    rng = np.random.default_rng(seed)
    c = synth.curve(rng, p, 9, 15, knots="random", min_gap=0.02)
    ctrl = c.ctrl.astype(np.float64)
    g = rng.normal(size=(len(c.u), 3))

    def L(pw):
        return float((O.curve_eval(p, c.U, _cart(pw), c.u) * g).sum())

    dpw = O.curve_vjp_homog(p, c.U, ctrl, c.u, g)
    _fd(L, _homog(ctrl), dpw)


def test_homogeneous_and_cartesian_gradients_are_one_chain_rule():
    # x = Pw.x / Pw.w, w = Pw.w: dL/dPw.xyz = dL/dx / w, dL/dPw.w = dL/dw - (x . dL/dx) / w
    rng = np.random.default_rng(6)
    s = synth.surface(rng, 3, 3, 8, 7, 9, 10, knots="random", min_gap=0.02)
    ctrl = s.ctrl.astype(np.float64)
    g = rng.normal(size=(len(s.u), len(s.v), 3))
    dc, _, _ = O.surface_vjp(s.p, s.q, s.U, s.V, ctrl, s.u, s.v, g, want_knots=False)
    dpw = O.surface_vjp_homog(s.p, s.q, s.U, s.V, ctrl, s.u, s.v, g)
    w = ctrl[..., 3:4]
    np.testing.assert_allclose(dpw[..., :3], dc[..., :3] / w, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(dpw[..., 3], dc[..., 3] - (ctrl[..., :3] * dc[..., :3]).sum(-1) / w[..., 0],
                               rtol=1e-10, atol=1e-13)
