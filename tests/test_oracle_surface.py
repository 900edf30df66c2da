"""Pins of the oracle's rational surface and curve evaluation (Eq. 3), its
gradients (Eq. 7, Eq. 8, Eq. 9 and the knot derivative of Sec. 3.2), the MSE loss
and the Adam step, against facts fixed by geometry, by library routines and by
central finite differences."""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_14547_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_surface(seed, p=3, q=2, n1=7, m1=6, nu=9, nv=8, knots="random"):
    rng = np.random.default_rng(seed)
    s = synth.surface(rng, p, q, n1, m1, nu, nv, knots=knots, min_gap=0.02)
    ctrl = s.ctrl.astype(np.float64)
    ctrl[..., :3] += rng.normal(0, 0.3, size=ctrl[..., :3].shape)
    return s.p, s.q, s.U.astype(np.float64), s.V.astype(np.float64), ctrl, s.u.astype(np.float64), s.v.astype(np.float64)


def test_endpoint_interpolation_clamped():
    p, q, U, V, ctrl, u, v = small_surface(1)
    S = O.surface_eval(p, q, U, V, ctrl, [0.0, 1.0], [0.0, 1.0])
    np.testing.assert_allclose(S[0, 0], ctrl[0, 0, :3], atol=1e-15)
    np.testing.assert_allclose(S[0, 1], ctrl[0, -1, :3], atol=1e-15)
    np.testing.assert_allclose(S[1, 0], ctrl[-1, 0, :3], atol=1e-15)
    np.testing.assert_allclose(S[1, 1], ctrl[-1, -1, :3], atol=1e-15)


def _decasteljau(points, t):
    pts = [np.array(x, dtype=np.float64) for x in points]
    while len(pts) > 1:
        pts = [(1 - t) * pts[i] + t * pts[i + 1] for i in range(len(pts) - 1)]
    return pts[0]


@pytest.mark.parametrize("p,q", [(1, 1), (2, 3), (3, 3), (4, 2), (5, 5)])
def test_bezier_patch_matches_de_casteljau(p, q):
    rng = np.random.default_rng(p * 7 + q)
    U = np.concatenate([np.zeros(p + 1), np.ones(p + 1)])
    V = np.concatenate([np.zeros(q + 1), np.ones(q + 1)])
    ctrl = np.concatenate([rng.normal(size=(p + 1, q + 1, 3)), rng.uniform(0.5, 2, size=(p + 1, q + 1, 1))], -1)
    Pw = np.concatenate([ctrl[..., :3] * ctrl[..., 3:], ctrl[..., 3:]], -1)  # homogeneous points
    u = rng.uniform(0, 1, 5)
    v = rng.uniform(0, 1, 4)
    S = O.surface_eval(p, q, U, V, ctrl, u, v)
    for a, ua in enumerate(u):
        for b, vb in enumerate(v):
            col = [_decasteljau(Pw[i], vb) for i in range(p + 1)]
            h = _decasteljau(col, ua)
            np.testing.assert_allclose(S[a, b], h[:3] / h[3], atol=1e-14)


def test_unit_weights_reduce_to_bspline_scipy():
    interp = pytest.importorskip("scipy.interpolate")
    p, q, U, V, ctrl, u, v = small_surface(3)
    ctrl[..., 3] = 1.0
    S = O.surface_eval(p, q, U, V, ctrl, u, v)
    Bu = interp.BSpline.design_matrix(u, U, p).toarray()
    Bv = interp.BSpline.design_matrix(v, V, q).toarray()
    ref = np.einsum("ai,ijc,bj->abc", Bu, ctrl[..., :3], Bv)
    np.testing.assert_allclose(S, ref, atol=1e-14)


def test_weight_scaling_invariance_and_affine_invariance():
    p, q, U, V, ctrl, u, v = small_surface(4)
    S = O.surface_eval(p, q, U, V, ctrl, u, v)
    c2 = ctrl.copy()
    c2[..., 3] *= 3.7
    np.testing.assert_allclose(O.surface_eval(p, q, U, V, c2, u, v), S, atol=1e-14)
    rng = np.random.default_rng(5)
    A = rng.normal(size=(3, 3))
    t = rng.normal(size=3)
    c3 = ctrl.copy()
    c3[..., :3] = ctrl[..., :3] @ A.T + t
    np.testing.assert_allclose(O.surface_eval(p, q, U, V, c3, u, v), S @ A.T + t, atol=1e-13)


def test_rational_circles_are_exact():
    g = json.load(open(os.path.join(GOLDEN, "rational_circle.json")))
    uu = np.linspace(0, 1, 101)
    for key in ("quarter_circle", "full_circle"):
        c = g[key]
        C = O.curve_eval(c["p"], c["U"], c["ctrl"], uu)
        np.testing.assert_allclose(np.linalg.norm(C, axis=1), 1.0, atol=1e-15)
        np.testing.assert_allclose(C[:, 2], 0.0, atol=0)
    # the full circle passes its four axis points at the double knots
    c = g["full_circle"]
    C = O.curve_eval(c["p"], c["U"], c["ctrl"], [0.25, 0.5, 0.75])
    np.testing.assert_allclose(C, [[0, 1, 0], [-1, 0, 0], [0, -1, 0]], atol=1e-15)
    # cylinder = circle (u) x line (v)
    cy = g["cylinder"]
    circ = np.array(c["ctrl"], dtype=np.float64)
    net = np.zeros((len(circ), 2, 4))
    for j, z in enumerate((0.0, 1.0)):
        net[:, j, :] = circ
        net[:, j, 2] = z
    vv = np.linspace(0, 1, 7)
    S = O.surface_eval(2, cy["q"], c["U"], cy["V"], net, uu, vv)
    np.testing.assert_allclose(np.linalg.norm(S[..., :2], axis=-1), 1.0, atol=1e-15)
    np.testing.assert_allclose(S[..., 2], np.broadcast_to(vv, S.shape[:2]), atol=1e-15)


def _boehm_insert(p, U, Pw, t):
    """Insert knot t once into a curve with homogeneous control points Pw (rows)."""
    n1 = len(Pw)
    k = int(np.searchsorted(U, t, side="right") - 1)
    new = np.zeros((n1 + 1,) + Pw.shape[1:])
    for i in range(n1 + 1):
        if i <= k - p:
            new[i] = Pw[i]
        elif i >= k + 1:
            new[i] = Pw[i - 1]
        else:
            a = (t - U[i]) / (U[i + p] - U[i])
            new[i] = a * Pw[i] + (1 - a) * Pw[i - 1]
    return np.insert(U, k + 1, t), new


def test_knot_insertion_invariance():
    p, q, U, V, ctrl, u, v = small_surface(6)
    Pw = np.concatenate([ctrl[..., :3] * ctrl[..., 3:], ctrl[..., 3:]], -1)
    U2, Pw2 = _boehm_insert(p, U, Pw, 0.4321)
    ctrl2 = np.concatenate([Pw2[..., :3] / Pw2[..., 3:], Pw2[..., 3:]], -1)
    np.testing.assert_allclose(O.surface_eval(p, q, U2, V, ctrl2, u, v), O.surface_eval(p, q, U, V, ctrl, u, v), atol=1e-13)


# ------------------------------------------------------------- gradients (FD)
def _fd_check(f, x, grad, idxs, h, rtol):
    for idx in idxs:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (f(xp) - f(xm)) / (2 * h)
        scale = max(abs(fd), abs(grad[idx]), 1e-3)
        assert abs(fd - grad[idx]) <= rtol * scale, (idx, fd, grad[idx])


@pytest.mark.parametrize("seed,p,q", [(10, 3, 3), (11, 2, 4), (12, 1, 2), (13, 5, 3)])
def test_surface_gradients_central_differences(seed, p, q):
    _, _, U, V, ctrl, u, v = small_surface(seed, p=p, q=q, n1=p + 5, m1=q + 4, nu=11, nv=10)
    rng = np.random.default_rng(seed)
    g = rng.normal(size=(len(u), len(v), 3))
    dctrl, dU, dV = O.surface_vjp(p, q, U, V, ctrl, u, v, g)
    L = lambda c, UU=U, VV=V: float((O.surface_eval(p, q, UU, VV, c, u, v) * g).sum())
    idxs = [(int(rng.integers(0, ctrl.shape[0])), int(rng.integers(0, ctrl.shape[1])), c) for c in range(4) for _ in range(4)]
    _fd_check(L, ctrl, dctrl, idxs, 1e-6, 1e-6)
    # interior knots only (end knots carry no gradient by the fixed-domain reading)
    for k in range(p + 1, len(U) - p - 1):
        _fd_check(lambda UU: L(ctrl, UU, V), U, dU, [k], 1e-7, 1e-6)
    for k in range(q + 1, len(V) - q - 1):
        _fd_check(lambda VV: L(ctrl, U, VV), V, dV, [k], 1e-7, 1e-6)
    assert np.all(dU[: p + 1] == 0) and np.all(dU[len(U) - p - 1:] == 0)
    assert np.all(dV[: q + 1] == 0) and np.all(dV[len(V) - q - 1:] == 0)


@pytest.mark.parametrize("seed,p", [(20, 3), (21, 2), (22, 5)])
def test_curve_gradients_central_differences(seed, p):
    rng = np.random.default_rng(seed)
    c = synth.curve(rng, p, p + 8, 37, min_gap=0.02)
    U, ctrl, u = c.U.astype(np.float64), c.ctrl.astype(np.float64), c.u.astype(np.float64)
    g = rng.normal(size=(len(u), 3))
    dctrl, dU = O.curve_vjp(p, U, ctrl, u, g)
    L = lambda cc, UU=U: float((O.curve_eval(p, UU, cc, u) * g).sum())
    idxs = [(int(rng.integers(0, ctrl.shape[0])), cc) for cc in range(4) for _ in range(4)]
    _fd_check(L, ctrl, dctrl, idxs, 1e-6, 1e-6)
    for k in range(p + 1, len(U) - p - 1):
        _fd_check(lambda UU: L(ctrl, UU), U, dU, [k], 1e-7, 1e-6)


def test_curve_equals_degenerate_surface():
    # a curve is a surface with one control column, degree 0 in v and one sample
    rng = np.random.default_rng(30)
    c = synth.curve(rng, 3, 12, 40)
    S = O.surface_eval(3, 0, c.U, [0.0, 1.0], c.ctrl[:, None, :], c.u, [0.5])
    np.testing.assert_allclose(S[:, 0, :], O.curve_eval(3, c.U, c.ctrl, c.u), atol=1e-15)
    g = rng.normal(size=(len(c.u), 3))
    dcs, dUs, _ = O.surface_vjp(3, 0, c.U, [0.0, 1.0], c.ctrl[:, None, :], c.u, [0.5], g[:, None, :])
    dcc, dUc = O.curve_vjp(3, c.U, c.ctrl, c.u, g)
    np.testing.assert_allclose(dcs[:, 0, :], dcc, atol=1e-13)
    np.testing.assert_allclose(dUs, dUc, atol=1e-12)


def test_mse_gradient_central_differences():
    rng = np.random.default_rng(40)
    S = rng.normal(size=(5, 6, 3))
    T = rng.normal(size=(5, 6, 3))
    L, g = O.mse(S, T, S.size)
    np.testing.assert_allclose(L, np.mean((S - T) ** 2), rtol=1e-14)
    h = 1e-6
    for idx in [(0, 0, 0), (4, 5, 2), (2, 3, 1)]:
        Sp, Sm = S.copy(), S.copy()
        Sp[idx] += h
        Sm[idx] -= h
        fd = (O.mse(Sp, T, S.size)[0] - O.mse(Sm, T, S.size)[0]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-8


def test_adam_matches_torch_optim():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(50)
    theta0 = rng.normal(size=37)
    grads = [rng.normal(size=37) for _ in range(5)]
    p = torch.nn.Parameter(torch.tensor(theta0, dtype=torch.float64))
    opt = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    th, m, v = theta0.copy(), np.zeros(37), np.zeros(37)
    for t, g in enumerate(grads, start=1):
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        th, m, v = O.adam(th, g, m, v, t, lr=1e-2)
        np.testing.assert_allclose(th, p.detach().numpy(), rtol=0, atol=1e-13)
