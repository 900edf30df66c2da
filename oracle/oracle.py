"""Python access to the FP64 CPU oracle (``nurbs_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and by
the CPU-baseline leg of the benchmark.  The product path never imports it.  It
shares no code with the CUDA library.

Each function takes numpy arrays, widens them to float64 (exact for the FP32
inputs the GPU path sees) and calls the C routine of the same role:

* ``find_span``, ``basis_funs``        -- span search and nonzero basis (Sec. 3.1 steps 1-2)
* ``basis_cox_de_boor``               -- brute-force recursion, Eq. 4 / Eq. 5
* ``basis_knot_jac``                  -- knot Jacobian of the nonzero basis (Sec. 3.2)
* ``basis_knot_jac_sigma``            -- the same with the Gaussian-smoothed indicator term
* ``surface_eval`` / ``curve_eval``   -- Eq. 3 (and its one-direction form)
* ``surface_vjp`` / ``curve_vjp``     -- Eq. 7, Eq. 8, Eq. 9 + knot derivative
* ``surface_vjp_homog`` / ``curve_vjp_homog`` -- gradient w.r.t. homogeneous Pw (Eq. 3)
* ``basis_ders``                      -- u-derivative of the nonzero basis (of Eq. 4)
* ``surface_derivs`` / ``curve_derivs`` -- tangents S_u, S_v, unit normals (curve: C')
* ``mse``, ``adam``                   -- the L2 (MSE) loss and the Adam step of Sec. 4
* ``nearest``, ``chamfer``            -- Chamfer and Hausdorff distances of Sec. 4 (numpy)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nurbs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libnurbs_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build (plain C, no CUDA)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i, d, sz = ctypes.c_int, ctypes.c_double, ctypes.c_size_t
            L.nurbs_oracle_find_span.argtypes = [i, i, d, _D]
            L.nurbs_oracle_find_span.restype = i
            L.nurbs_oracle_basis_funs.argtypes = [i, d, i, _D, _D]
            L.nurbs_oracle_basis_cox_de_boor.argtypes = [i, i, d, _D, i]
            L.nurbs_oracle_basis_cox_de_boor.restype = d
            L.nurbs_oracle_basis_knot_jac.argtypes = [i, d, i, _D, _D, _D]
            L.nurbs_oracle_surface_eval.argtypes = [i, i, i, i, _D, _D, _D, i, _D, i, _D, _D]
            L.nurbs_oracle_surface_vjp.argtypes = [i, i, i, i, _D, _D, _D, i, _D, i, _D, _D, _D, _D, _D]
            L.nurbs_oracle_surface_vjp_sigma.argtypes = [i, i, i, i, _D, _D, _D, i, _D, i, _D, _D, _D, _D, _D, d]
            L.nurbs_oracle_curve_vjp_sigma.argtypes = [i, i, _D, _D, i, _D, _D, _D, _D, d]
            L.nurbs_oracle_basis_knot_jac_sigma.argtypes = [i, d, i, _D, d, _D, _D]
            L.nurbs_oracle_curve_eval.argtypes = [i, i, _D, _D, i, _D, _D]
            L.nurbs_oracle_curve_vjp.argtypes = [i, i, _D, _D, i, _D, _D, _D, _D]
            L.nurbs_oracle_surface_vjp_homog.argtypes = [i, i, i, i, _D, _D, _D, i, _D, i, _D, _D, _D]
            L.nurbs_oracle_curve_vjp_homog.argtypes = [i, i, _D, _D, i, _D, _D, _D]
            L.nurbs_oracle_basis_ders.argtypes = [i, d, i, _D, _D]
            L.nurbs_oracle_surface_derivs.argtypes = [i, i, i, i, _D, _D, _D, i, _D, i, _D, _D, _D, _D, _D]
            L.nurbs_oracle_curve_derivs.argtypes = [i, i, _D, _D, i, _D, _D, _D]
            L.nurbs_oracle_mse.argtypes = [sz, _D, _D, d, _D]
            L.nurbs_oracle_mse.restype = d
            L.nurbs_oracle_adam.argtypes = [sz, _D, _D, _D, _D, i, d, d, d, d]
            _lib = L
    return _lib


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(_D)


# --------------------------------------------------------------------- basis
def find_span(n: int, p: int, u: float, U) -> int:
    U = _f64(U)
    return int(lib().nurbs_oracle_find_span(n, p, float(u), _p(U)))


def basis_funs(span: int, u: float, p: int, U) -> np.ndarray:
    U = _f64(U)
    N = np.zeros(p + 1)
    lib().nurbs_oracle_basis_funs(span, float(u), p, _p(U), _p(N))
    return N


def basis_cox_de_boor(i: int, p: int, u: float, U) -> float:
    U = _f64(U)
    return float(lib().nurbs_oracle_basis_cox_de_boor(i, p, float(u), _p(U), len(U)))


def basis_knot_jac(span: int, u: float, p: int, U):
    """(N[p+1], dN[p+1, 2p]) with dN[r, k] = dN_{span-p+r}/dU[span-p+1+k]."""
    U = _f64(U)
    N = np.zeros(p + 1)
    dN = np.zeros((p + 1) * max(2 * p, 1))
    lib().nurbs_oracle_basis_knot_jac(span, float(u), p, _p(U), _p(N), _p(dN))
    return N, dN.reshape(p + 1, max(2 * p, 1))[:, : 2 * p]


def basis_knot_jac_sigma(span: int, u: float, p: int, U, sigma: float):
    """(N[p+1], J[p+1, 2p+2]) with J[r, k] = dN_{span-p+r}/dU[span-p+k] including
    the Gaussian-smoothed indicator term of bandwidth sigma (Sec. 3.2)."""
    U = _f64(U)
    N = np.zeros(p + 1)
    J = np.zeros((p + 1) * (2 * p + 2))
    lib().nurbs_oracle_basis_knot_jac_sigma(span, float(u), p, _p(U), float(sigma), _p(N), _p(J))
    return N, J.reshape(p + 1, 2 * p + 2)


# ------------------------------------------------------------------- surface
def surface_eval(p, q, U, V, ctrl, u, v) -> np.ndarray:
    """ctrl: [n1, m1, 4] (x, y, z, w).  Returns S[nu, nv, 3] in float64."""
    ctrl = _f64(ctrl)
    n1, m1 = ctrl.shape[0], ctrl.shape[1]
    U, V, u, v = _f64(U), _f64(V), _f64(u), _f64(v)
    assert len(U) == n1 + p + 1 and len(V) == m1 + q + 1
    out = np.zeros((len(u), len(v), 3))
    lib().nurbs_oracle_surface_eval(p, q, n1, m1, _p(U), _p(V), _p(ctrl), len(u), _p(u), len(v), _p(v), _p(out))
    return out


def surface_vjp(p, q, U, V, ctrl, u, v, g, want_ctrl=True, want_knots=True, knot_sigma=0.0):
    """Returns (dctrl[n1, m1, 4], dU, dV); entries not requested are None.
    knot_sigma > 0 takes the knot derivative in its Gaussian-smoothed form."""
    ctrl = _f64(ctrl)
    n1, m1 = ctrl.shape[0], ctrl.shape[1]
    U, V, u, v, g = _f64(U), _f64(V), _f64(u), _f64(v), _f64(g)
    assert g.shape == (len(u), len(v), 3)
    dctrl = np.zeros((n1, m1, 4)) if want_ctrl else None
    dU = np.zeros(len(U)) if want_knots else None
    dV = np.zeros(len(V)) if want_knots else None
    lib().nurbs_oracle_surface_vjp_sigma(p, q, n1, m1, _p(U), _p(V), _p(ctrl), len(u), _p(u), len(v), _p(v),
                                         _p(g), _p(dctrl), _p(dU), _p(dV), float(knot_sigma))
    return dctrl, dU, dV


def surface_vjp_homog(p, q, U, V, ctrl, u, v, g):
    """dL/dPw[n1, m1, 4] for the homogeneous control points Pw = (w x, w y, w z, w)."""
    ctrl = _f64(ctrl)
    n1, m1 = ctrl.shape[0], ctrl.shape[1]
    U, V, u, v, g = _f64(U), _f64(V), _f64(u), _f64(v), _f64(g)
    assert g.shape == (len(u), len(v), 3)
    dpw = np.zeros((n1, m1, 4))
    lib().nurbs_oracle_surface_vjp_homog(p, q, n1, m1, _p(U), _p(V), _p(ctrl), len(u), _p(u), len(v), _p(v),
                                         _p(g), _p(dpw))
    return dpw


# --------------------------------------------------------------------- curve
def curve_eval(p, U, ctrl, u) -> np.ndarray:
    ctrl = _f64(ctrl)
    n1 = ctrl.shape[0]
    U, u = _f64(U), _f64(u)
    assert len(U) == n1 + p + 1
    out = np.zeros((len(u), 3))
    lib().nurbs_oracle_curve_eval(p, n1, _p(U), _p(ctrl), len(u), _p(u), _p(out))
    return out


def curve_vjp(p, U, ctrl, u, g, want_ctrl=True, want_knots=True, knot_sigma=0.0):
    ctrl = _f64(ctrl)
    n1 = ctrl.shape[0]
    U, u, g = _f64(U), _f64(u), _f64(g)
    dctrl = np.zeros((n1, 4)) if want_ctrl else None
    dU = np.zeros(len(U)) if want_knots else None
    lib().nurbs_oracle_curve_vjp_sigma(p, n1, _p(U), _p(ctrl), len(u), _p(u), _p(g), _p(dctrl), _p(dU),
                                       float(knot_sigma))
    return dctrl, dU


def curve_vjp_homog(p, U, ctrl, u, g):
    ctrl = _f64(ctrl)
    n1 = ctrl.shape[0]
    U, u, g = _f64(U), _f64(u), _f64(g)
    dpw = np.zeros((n1, 4))
    lib().nurbs_oracle_curve_vjp_homog(p, n1, _p(U), _p(ctrl), len(u), _p(u), _p(g), _p(dpw))
    return dpw


# ----------------------------------------------------------------- loss, adam

def basis_ders(span: int, u: float, p: int, U) -> np.ndarray:
    """dN_{span-p+r}(u)/du, r = 0..p (the u-derivative of Eq. 4)."""
    U = _f64(U)
    dN = np.zeros(p + 1)
    lib().nurbs_oracle_basis_ders(span, float(u), p, _p(U), _p(dN))
    return dN


def surface_derivs(p, q, U, V, ctrl, u, v):
    """Points, tangents S_u, S_v and unit normals, each [nu, nv, 3]."""
    U, V, ctrl, u, v = _f64(U), _f64(V), _f64(ctrl), _f64(u), _f64(v)
    n1, m1 = ctrl.shape[0], ctrl.shape[1]
    outs = [np.zeros((len(u), len(v), 3)) for _ in range(4)]
    lib().nurbs_oracle_surface_derivs(p, q, n1, m1, _p(U), _p(V), _p(ctrl), len(u), _p(u), len(v), _p(v),
                                      *[_p(x) for x in outs])
    return tuple(outs)


def curve_derivs(p, U, ctrl, u):
    """Points and tangents C'(u), each [nu, 3]."""
    U, ctrl, u = _f64(U), _f64(ctrl), _f64(u)
    C, Cu = np.zeros((len(u), 3)), np.zeros((len(u), 3))
    lib().nurbs_oracle_curve_derivs(p, ctrl.shape[0], _p(U), _p(ctrl), len(u), _p(u), _p(C), _p(Cu))
    return C, Cu

def mse(S, T, count: float):
    """(L, g): L = sum (S-T)^2 / count, g = 2 (S-T) / count."""
    S, T = _f64(S), _f64(T)
    g = np.zeros_like(S)
    L = lib().nurbs_oracle_mse(S.size, _p(S), _p(T), float(count), _p(g))
    return float(L), g


def adam(theta, g, m, v, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step; returns updated copies (theta, m, v)."""
    theta, g, m, v = _f64(theta).copy(), _f64(g), _f64(m).copy(), _f64(v).copy()
    lib().nurbs_oracle_adam(theta.size, _p(theta), _p(g), _p(m), _p(v), int(t), lr, b1, b2, eps)
    return theta, m, v


# ------------------------------------------------------- point-set distances
def _d2_f32(A, B):
    """Squared distances in float32, each as ((dx*dx + dy*dy) + dz*dz) with
    every operation rounded separately: the precision the argmin is decided in."""
    A32, B32 = np.asarray(A, np.float32), np.asarray(B, np.float32)
    d = A32[:, None, :] - B32[None, :, :]
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def nearest(A, B):
    """For every point of A: index of its nearest point of B (the first one on
    ties, decided on float32 squared distances) and the FP64 distance to it."""
    A, B = np.asarray(A, np.float64).reshape(-1, 3), np.asarray(B, np.float64).reshape(-1, 3)
    if len(A) == 0 or len(B) == 0:
        return np.full(len(A), -1, np.int64), np.zeros(len(A))
    nn = np.argmin(_d2_f32(A, B), axis=1)
    return nn, np.linalg.norm(A - B[nn], axis=1)


def chamfer(P, Q):
    """The paper's point-set losses (Sec. 4): Chamfer distance
    L_CD = sum_i min_j |P_i - Q_j| + sum_j min_i |P_i - Q_j| and Hausdorff distance
    L_HD = max_i min_j |P_i - Q_j| + max_j min_i |P_i - Q_j|, with their gradients
    with respect to P.  Returns (cd, hd, grad_cd[nP, 3], grad_hd[nP, 3], nn_p, nn_q).
    A zero distance contributes no gradient; ties in argmax take the first index;
    an empty set gives 0 and zero gradients."""
    P, Q = np.asarray(P, np.float64).reshape(-1, 3), np.asarray(Q, np.float64).reshape(-1, 3)
    gcd, ghd = np.zeros_like(P), np.zeros_like(P)
    nn_p, d_p = nearest(P, Q)
    nn_q, d_q = nearest(Q, P)
    if len(P) == 0 or len(Q) == 0:
        return 0.0, 0.0, gcd, ghd, nn_p, nn_q
    cd = d_p.sum() + d_q.sum()
    hd = d_p.max() + d_q.max()
    for i in range(len(P)):
        if d_p[i] > 0:
            gcd[i] += (P[i] - Q[nn_p[i]]) / d_p[i]
    for j in range(len(Q)):
        if d_q[j] > 0:
            gcd[nn_q[j]] += (P[nn_q[j]] - Q[j]) / d_q[j]
    i_star, j_star = int(np.argmax(d_p)), int(np.argmax(d_q))
    if d_p[i_star] > 0:
        ghd[i_star] += (P[i_star] - Q[nn_p[i_star]]) / d_p[i_star]
    if d_q[j_star] > 0:
        ghd[nn_q[j_star]] += (P[nn_q[j_star]] - Q[j_star]) / d_q[j_star]
    return float(cd), float(hd), gcd, ghd, nn_p, nn_q
