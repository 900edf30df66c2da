"""Pins of the oracle's parametric derivatives: the u-derivative of the basis
(of Eq. 4), surface tangents S_u, S_v and unit normals, curve tangents.

They are checked against:
- finite differences of the independently pinned forward;
- the Bernstein derivative closed form;
- the vanishing derivative of the partition of unity;
- circle, cylinder and plane geometry.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_14547_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _knots(seed, p, n1):
    rng = np.random.default_rng(seed)
    return synth.clamped_random_knots(rng, n1, p, min_gap=0.03).astype(np.float64)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_basis_derivative_matches_central_differences(p):
    U = _knots(p, p, 10)
    n = 9
    nk = len(U)
    rng = np.random.default_rng(100 + p)
    for u in rng.uniform(0.01, 0.99, size=40):
        s = O.find_span(n, p, u, U)
        # keep the stencil inside one span (the basis is a polynomial there)
        h = 1e-6
        if not (U[s] < u - h and u + h < U[s + 1]):
            continue
        dN = O.basis_ders(s, u, p, U)
        for r in range(p + 1):
            i = s - p + r
            fd = (O.basis_cox_de_boor(i, p, u + h, U) - O.basis_cox_de_boor(i, p, u - h, U)) / (2 * h)
            assert abs(dN[r] - fd) <= 1e-6 * max(1.0, abs(fd)), (p, u, r, dN[r], fd)
        # partition of unity: the derivatives of the nonzero functions sum to 0
        assert abs(dN.sum()) <= 1e-12 * max(1.0, np.abs(dN).max())


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_bernstein_derivative_closed_form(p):
    U = np.array([0.0] * (p + 1) + [1.0] * (p + 1))

    def bern(k, d, t):
        if k < 0 or k > d:
            return 0.0
        return math.comb(d, k) * t ** k * (1 - t) ** (d - k)

    for t in np.linspace(0.0, 1.0, 11):
        s = O.find_span(p, p, t, U)
        dN = O.basis_ders(s, t, p, U)
        want = [p * (bern(k - 1, p - 1, t) - bern(k, p - 1, t)) for k in range(p + 1)]
        np.testing.assert_allclose(dN, want, rtol=0, atol=1e-12)


def _rand_surface(seed, p=3, q=2):
    rng = np.random.default_rng(seed)
    s = synth.surface(rng, p, q, 8, 7, 9, 11, knots="random", min_gap=0.03)
    ctrl = s.ctrl.astype(np.float64)
    ctrl[..., :3] += rng.normal(0, 0.3, size=ctrl[..., :3].shape)
    return s.p, s.q, s.U.astype(np.float64), s.V.astype(np.float64), ctrl


@pytest.mark.parametrize("seed,p,q", [(0, 3, 2), (1, 2, 4), (2, 5, 1)])
def test_surface_tangents_and_normals_match_differences(seed, p, q):
    p, q, U, V, ctrl = _rand_surface(seed, p, q)
    rng = np.random.default_rng(200 + seed)
    u = np.sort(rng.uniform(0.02, 0.98, 6))
    v = np.sort(rng.uniform(0.02, 0.98, 5))
    S, Su, Sv, Nrm = O.surface_derivs(p, q, U, V, ctrl, u, v)
    np.testing.assert_allclose(S, O.surface_eval(p, q, U, V, ctrl, u, v), rtol=0, atol=1e-14)
    h = 1e-6
    fu = (O.surface_eval(p, q, U, V, ctrl, u + h, v) - O.surface_eval(p, q, U, V, ctrl, u - h, v)) / (2 * h)
    fv = (O.surface_eval(p, q, U, V, ctrl, u, v + h) - O.surface_eval(p, q, U, V, ctrl, u, v - h)) / (2 * h)
    # stencils that straddle a knot see the one-sided derivative: drop them
    def inside(x, K):
        return np.array([not np.any(np.abs(K - t) <= 2 * h) for t in x])

    mu, mv = inside(u, U), inside(v, V)
    sel = np.ix_(mu, mv)
    scale = np.abs(Su).max() + np.abs(Sv).max()
    np.testing.assert_allclose(Su[sel], fu[sel], rtol=0, atol=1e-6 * scale)
    np.testing.assert_allclose(Sv[sel], fv[sel], rtol=0, atol=1e-6 * scale)
    cr = np.cross(fu, fv)
    cr /= np.linalg.norm(cr, axis=-1, keepdims=True)
    np.testing.assert_allclose(Nrm[sel], cr[sel], rtol=0, atol=1e-6)
    np.testing.assert_allclose(np.linalg.norm(Nrm, axis=-1), 1.0, atol=1e-12)


def test_curve_tangent_matches_differences_and_degenerate_surface():
    rng = np.random.default_rng(7)
    c = synth.curve(rng, 4, 12, 9, min_gap=0.03)
    U, ctrl = c.U.astype(np.float64), c.ctrl.astype(np.float64)
    u = np.sort(rng.uniform(0.02, 0.98, 9))
    C, Cu = O.curve_derivs(4, U, ctrl, u)
    h = 1e-6
    fd = (O.curve_eval(4, U, ctrl, u + h) - O.curve_eval(4, U, ctrl, u - h)) / (2 * h)
    keep = np.array([not np.any(np.abs(U - t) <= 2 * h) for t in u])
    np.testing.assert_allclose(Cu[keep], fd[keep], rtol=0, atol=1e-6 * np.abs(Cu).max())
    # a curve is the surface with a degree-1 line of identical rows in v
    net = np.stack([ctrl, ctrl], axis=1)
    S, Su, Sv, _ = O.surface_derivs(4, 1, U, [0, 0, 1, 1], net, u, [0.3])
    np.testing.assert_allclose(S[:, 0], C, atol=1e-14)
    np.testing.assert_allclose(Su[:, 0], Cu, atol=1e-12 * np.abs(Cu).max())
    np.testing.assert_allclose(Sv, 0.0, atol=1e-12)


def test_circle_tangent_and_cylinder_normal():
    g = json.load(open(os.path.join(GOLDEN, "rational_circle.json")))
    uu = np.linspace(0.0, 1.0, 41)
    for key in ("quarter_circle", "full_circle"):
        c = g[key]
        C, Cu = O.curve_derivs(c["p"], c["U"], c["ctrl"], uu)
        # a circle's tangent is perpendicular to its radius and never vanishes
        np.testing.assert_allclose(np.einsum("ij,ij->i", C, Cu), 0.0, atol=1e-13)
        assert np.linalg.norm(Cu, axis=1).min() > 0.5
        np.testing.assert_allclose(Cu[:, 2], 0.0, atol=0)
    c, cy = g["full_circle"], g["cylinder"]
    circ = np.array(c["ctrl"], dtype=np.float64)
    net = np.zeros((len(circ), 2, 4))
    for j, z in enumerate((0.0, 1.0)):
        net[:, j, :] = circ
        net[:, j, 2] = z
    vv = np.linspace(0.0, 1.0, 5)
    S, Su, Sv, Nrm = O.surface_derivs(2, cy["q"], c["U"], cy["V"], net, uu, vv)
    # along the line direction the tangent is (0, 0, 1); the normal is radial
    np.testing.assert_allclose(Sv, np.broadcast_to([0.0, 0.0, 1.0], Sv.shape), atol=1e-14)
    radial = S.copy()
    radial[..., 2] = 0.0
    np.testing.assert_allclose(np.abs(np.einsum("abk,abk->ab", Nrm, radial)), 1.0, atol=1e-12)


def test_plane_normal_is_constant():
    rng = np.random.default_rng(11)
    s = synth.surface(rng, 3, 3, 7, 6, 8, 8, knots="random", min_gap=0.03)
    ctrl = s.ctrl.astype(np.float64)
    ctrl[..., 2] = 0.4              # every control point in the plane z = 0.4
    S, Su, Sv, Nrm = O.surface_derivs(3, 3, s.U, s.V, ctrl, s.u, s.v)
    np.testing.assert_allclose(S[..., 2], 0.4, atol=1e-15)
    np.testing.assert_allclose(np.abs(Nrm[..., 2]), 1.0, atol=1e-12)
    np.testing.assert_allclose(Su[..., 2], 0.0, atol=1e-13)
