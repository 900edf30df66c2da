"""Pins of the oracle's knot derivative in the paper's Gaussian-smoothed form
(Sec. 3.2).  The degree-0 indicator's knot derivative is -G(u - U_j) at its left
knot and +G(u - U_{j+1}) at its right knot.  It is pushed through the full
Cox-de Boor triangle.

- As sigma -> 0 the Jacobian equals the almost-everywhere one.
- Its coefficient part equals the independent nonzero-triangle Jacobian.
- Its indicator part equals an independent computation: the triangle is linear in
  the degree-0 values when its coefficients are frozen, so the part is that map
  applied to the central differences of the smoothed indicators Phi((u-U_j)/s) -
  Phi((u-U_{j+1})/s).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_14547_gb300 import synth


def _phi(x):
    return 0.5 * (1.0 + math.erf(x / math.sqrt(2.0)))


def _frozen_map(span, u, p, U):
    """M[r, j]: N^p_{span-p+r}(u) when the degree-0 values are the unit vector
    e_j (j over span-p .. span+p) and every coefficient of Eq. 4 keeps its value
    at the given knots (0/0 := 0).  Plain recursion, level by level."""
    lo, width = span - p, 2 * p + 1
    M = np.zeros((p + 1, width))
    for j in range(width):
        val = [1.0 if t == j else 0.0 for t in range(width)]
        for d in range(1, p + 1):
            nxt = []
            for i in range(lo, span + p - d + 1):
                ad, bd = U[i + d] - U[i], U[i + d + 1] - U[i + 1]
                a = (u - U[i]) / ad if ad != 0 else 0.0
                b = (U[i + d + 1] - u) / bd if bd != 0 else 0.0
                nxt.append(a * val[i - lo] + b * val[i - lo + 1])
            val = nxt
        M[:, j] = val[: p + 1]
    return M


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_sigma_to_zero_matches_almost_everywhere_jacobian(p):
    rng = np.random.default_rng(300 + p)
    U = synth.clamped_random_knots(rng, 12, p, min_gap=0.03).astype(np.float64)
    for u in rng.uniform(0.02, 0.98, 15):
        s = O.find_span(11, p, u, U)
        N0, J0 = O.basis_knot_jac(s, u, p, U)
        Ns, Js = O.basis_knot_jac_sigma(s, u, p, U, 1e-9)
        np.testing.assert_allclose(Ns, N0, atol=1e-15)
        np.testing.assert_allclose(Js[:, 1:-1], J0, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(Js[:, [0, -1]], 0.0, atol=1e-300)
        # sigma = 0 exactly: the same coefficient part through the full triangle
        _, Jz = O.basis_knot_jac_sigma(s, u, p, U, 0.0)
        np.testing.assert_allclose(Jz[:, 1:-1], J0, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_indicator_part_matches_frozen_map_of_smoothed_indicators(p):
    rng = np.random.default_rng(400 + p)
    U = synth.clamped_random_knots(rng, 10, p, min_gap=0.05).astype(np.float64)
    sigma = 0.01
    checked = 0
    for k0 in range(p + 1, 10):                      # samples close to interior knots
        for off in (-0.6, -0.2, 0.15, 0.5):
            u = U[k0] + off * sigma
            s = O.find_span(9, p, u, U)
            _, Js = O.basis_knot_jac_sigma(s, u, p, U, sigma)
            _, Jz = O.basis_knot_jac_sigma(s, u, p, U, 0.0)
            M = _frozen_map(s, u, p, U)
            lo = s - p
            want = np.zeros((p + 1, 2 * p + 2))
            h = 1e-7
            for k in range(2 * p + 2):               # knot lo + k
                kk = lo + k
                dind = np.zeros(2 * p + 1)
                for j in range(2 * p + 1):           # degree-0 function lo + j
                    jj = lo + j
                    if kk not in (jj, jj + 1):
                        continue

                    def smooth(shift):
                        Ut = U.copy()
                        Ut[kk] += shift
                        return _phi((u - Ut[jj]) / sigma) - _phi((u - Ut[jj + 1]) / sigma)

                    dind[j] = (smooth(h) - smooth(-h)) / (2 * h)
                want[:, k] = M @ dind
            got = Js - Jz
            assert np.abs(got - want).max() <= 1e-5 * max(1.0, np.abs(want).max()), (p, k0, off)
            checked += 1
    assert checked >= 8


def test_sigma_vjp_tiny_sigma_and_far_samples():
    rng = np.random.default_rng(500)
    s = synth.surface(rng, 3, 2, 8, 7, 9, 11, knots="random", min_gap=0.03)
    g = rng.normal(size=(9, 11, 3))
    d0 = O.surface_vjp(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v, g)
    dt = O.surface_vjp(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v, g, knot_sigma=1e-9)
    for a, b in zip(d0, dt):
        np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-12)
    c = synth.curve(rng, 3, 12, 50, min_gap=0.03)
    gc = rng.normal(size=(50, 3))
    e0 = O.curve_vjp(c.p, c.U, c.ctrl, c.u, gc)
    et = O.curve_vjp(c.p, c.U, c.ctrl, c.u, gc, knot_sigma=1e-9)
    for a, b in zip(e0, et):
        np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-12)
