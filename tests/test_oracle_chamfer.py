"""Pins of the oracle's Chamfer and Hausdorff distances (Sec. 4): a Python-loop
brute force, identity, symmetry, translation invariance, and central
differences of the Chamfer distance."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def _loops(P, Q):
    def directed(A, B):
        out = []
        for a in A:
            best = None
            for b in B:
                d = math.sqrt(sum((a[k] - b[k]) ** 2 for k in range(3)))
                best = d if best is None or d < best else best
            out.append(best)
        return out
    dp, dq = directed(P, Q), directed(Q, P)
    return sum(dp) + sum(dq), max(dp) + max(dq)


def test_matches_loops_on_small_sets():
    rng = np.random.default_rng(1)
    P, Q = rng.normal(size=(7, 3)), rng.normal(size=(5, 3))
    cd, hd, *_ = O.chamfer(P, Q)
    wcd, whd = _loops(P.tolist(), Q.tolist())
    assert abs(cd - wcd) <= 1e-12 and abs(hd - whd) <= 1e-12


def test_identity_symmetry_translation():
    rng = np.random.default_rng(2)
    P, Q = rng.normal(size=(40, 3)), rng.normal(size=(33, 3))
    cd, hd, gcd, ghd, _, _ = O.chamfer(P, P)
    assert cd == 0.0 and hd == 0.0 and not gcd.any() and not ghd.any()
    a = O.chamfer(P, Q)
    b = O.chamfer(Q, P)
    assert abs(a[0] - b[0]) <= 1e-12 and abs(a[1] - b[1]) <= 1e-12
    t = np.array([3.0, -1.5, 0.25])
    c = O.chamfer(P + t, Q + t)
    assert abs(a[0] - c[0]) <= 1e-9 and abs(a[1] - c[1]) <= 1e-9


def test_empty_sets():
    P = np.zeros((0, 3))
    Q = np.ones((4, 3))
    cd, hd, gcd, ghd, nn_p, nn_q = O.chamfer(P, Q)
    assert cd == 0.0 and hd == 0.0 and gcd.shape == (0, 3)
    assert np.all(nn_q == -1)


@pytest.mark.parametrize("seed", [3, 4])
def test_gradients_match_central_differences(seed):
    rng = np.random.default_rng(seed)
    P, Q = rng.normal(size=(12, 3)), rng.normal(size=(9, 3))
    cd, hd, gcd, ghd, _, _ = O.chamfer(P, Q)
    h = 1e-7
    for i in range(len(P)):
        for k in range(3):
            Pp, Pm = P.copy(), P.copy()
            Pp[i, k] += h
            Pm[i, k] -= h
            fp, fm = O.chamfer(Pp, Q), O.chamfer(Pm, Q)
            assert abs((fp[0] - fm[0]) / (2 * h) - gcd[i, k]) <= 1e-6
            assert abs((fp[1] - fm[1]) / (2 * h) - ghd[i, k]) <= 1e-6
