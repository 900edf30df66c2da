"""Pins of the oracle's span search and basis functions (Sec. 3.1 steps 1-2, Eq. 4,
Eq. 5, and the knot derivative of Sec. 3.2) against facts fixed by the
mathematics: a hand-worked example, closed forms, partition of unity, local
support, a library B-spline routine and finite differences."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def random_knots(rng, n1, p, repeat=False):
    k = n1 - p - 1
    inner = np.sort(rng.uniform(0, 1, size=k))
    if repeat and k >= 3:
        inner[1] = inner[2]  # a double interior knot
        if p >= 2 and k >= 5:
            inner[3] = inner[4] = inner[2] if k == 5 else inner[4]
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


def test_worked_example_golden():
    g = json.load(open(os.path.join(GOLDEN, "basis_worked_example.json")))
    U, p, u = g["U"], g["p"], g["u"]
    n = len(U) - p - 2
    s = O.find_span(n, p, u, U)
    assert s == g["span"]
    N = O.basis_funs(s, u, p, U)
    np.testing.assert_allclose(N, g["N"], rtol=0, atol=1e-15)
    full = [O.basis_cox_de_boor(i, p, u, U) for i in range(n + 1)]
    np.testing.assert_allclose(full[g["nonzero_first_index"]: g["nonzero_first_index"] + p + 1], g["N"], atol=1e-15)
    assert sum(abs(x) for i, x in enumerate(full) if not (2 <= i <= 4)) == 0.0


def test_uniform_cubic_closed_form():
    # unclamped integer knots: on span [k, k+1) with t = u - k the four cubic
    # blending functions are (1-t)^3/6, (3t^3-6t^2+4)/6, (-3t^3+3t^2+3t+1)/6, t^3/6
    U = np.arange(12, dtype=np.float64)
    p = 3
    rng = np.random.default_rng(1)
    for _ in range(50):
        k = int(rng.integers(3, 8))
        t = float(rng.uniform(0, 1))
        u = k + t
        s = O.find_span(len(U) - p - 2, p, u, U)
        assert s == k
        N = O.basis_funs(s, u, p, U)
        ref = [(1 - t) ** 3 / 6, (3 * t ** 3 - 6 * t ** 2 + 4) / 6, (-3 * t ** 3 + 3 * t ** 2 + 3 * t + 1) / 6, t ** 3 / 6]
        np.testing.assert_allclose(N, ref, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_bezier_is_bernstein(p):
    U = np.concatenate([np.zeros(p + 1), np.ones(p + 1)])
    for u in np.linspace(0, 1, 23):
        s = O.find_span(p, p, u, U)
        N = O.basis_funs(s, u, p, U)
        ref = [math.comb(p, r) * u ** r * (1 - u) ** (p - r) for r in range(p + 1)]
        np.testing.assert_allclose(N, ref, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("repeat", [False, True])
def test_partition_of_unity_nonneg_local_support(p, repeat):
    rng = np.random.default_rng(p * 10 + repeat)
    n1 = p + 6
    U = random_knots(rng, n1, p, repeat)
    n = n1 - 1
    us = np.concatenate([rng.uniform(0, 1, 40), U[p: n + 2], [0.0, 1.0]])
    for u in us:
        s = O.find_span(n, p, u, U)
        assert p <= s <= n
        assert U[s] <= u and (u < U[s + 1] or (s == n and u == U[n + 1]))
        N = O.basis_funs(s, u, p, U)
        assert abs(N.sum() - 1.0) < 1e-14
        assert (N >= -1e-15).all()
        full = np.array([O.basis_cox_de_boor(i, p, u, U) for i in range(n1)])
        ref = np.zeros(n1)
        ref[s - p: s + 1] = N
        np.testing.assert_allclose(full, ref, atol=1e-14)


def test_span_search_largest_k():
    # repeated knots: the span is the largest k with U[k] <= u, so the chosen span is never empty
    U = np.array([0, 0, 0, 0, 0.2, 0.2, 0.5, 0.5, 0.5, 0.8, 1, 1, 1, 1], dtype=np.float64)
    p = 3
    n = len(U) - p - 2
    for u in [0.0, 0.1, 0.2, 0.3, 0.5, 0.6, 0.8, 0.9, 0.999, 1.0]:
        s = O.find_span(n, p, u, U)
        expect = n if u >= U[n + 1] else int(np.searchsorted(U, u, side="right") - 1)
        assert s == expect
        assert U[s] < U[s + 1]


def test_against_scipy_bspline_design_matrix():
    interp = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(7)
    for p in (1, 2, 3, 4, 5):
        n1 = 12
        U = random_knots(rng, n1, p)
        x = np.sort(rng.uniform(0, 1, 60))
        D = interp.BSpline.design_matrix(x, U, p).toarray()
        for a, u in enumerate(x):
            s = O.find_span(n1 - 1, p, u, U)
            N = O.basis_funs(s, u, p, U)
            np.testing.assert_allclose(D[a, s - p: s + 1], N, atol=1e-13)
            assert abs(D[a].sum() - 1) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_knot_jacobian_central_differences(p):
    rng = np.random.default_rng(100 + p)
    n1 = p + 7
    U = random_knots(rng, n1, p)
    gaps = np.diff(U)
    h = 1e-7
    for _ in range(12):
        u = float(rng.uniform(0.02, 0.98))
        if np.min(np.abs(U - u)) < 1e-3:
            continue
        s = O.find_span(n1 - 1, p, u, U)
        N, dN = O.basis_knot_jac(s, u, p, U)
        np.testing.assert_allclose(N, O.basis_funs(s, u, p, U), atol=1e-15)
        for k in range(2 * p):
            idx = s - p + 1 + k
            Up, Um = U.copy(), U.copy()
            Up[idx] += h
            Um[idx] -= h
            fd = (O.basis_funs(s, u, p, Up) - O.basis_funs(s, u, p, Um)) / (2 * h)
            scale = max(1.0, np.abs(dN[:, k]).max())
            np.testing.assert_allclose(dN[:, k], fd, atol=1e-6 * scale, rtol=0)
        # the basis sums to one for any knots, so its knot derivative sums to zero
        np.testing.assert_allclose(dN.sum(axis=0), 0.0, atol=1e-12 * max(1.0, np.abs(dN).max()))
    assert gaps.max() > 0
