"""GPU gradients with respect to the homogeneous control points Pw
(nurbs_plan_set_grad_homogeneous) against the oracle, on every path that writes
control-point gradients: surface tiles (single- and multi-tile items), curve
kernels, long curves on the tile kernels and the fused MSE step; the fit step's
Adam update still acts on (P, w)."""
import numpy as np
import pytest
import torch

from gpu_util import G_TOL, pack, rel_inf
from oracle import oracle as O
from paper_2104_14547_gb300 import _lib, batch, synth

pytestmark = pytest.mark.gpu
SURF, CURVE = _lib.KIND_SURFACE, _lib.KIND_CURVE


def _surfaces(seed):
    rng = np.random.default_rng(seed)
    return [synth.surface(rng, p, q, n1, m1, nu, nv, knots="random", min_gap=0.01)
            for p, q, n1, m1, nu, nv in ((3, 3, 10, 9, 40, 37), (2, 4, 8, 11, 300, 90),
                                         (1, 2, 6, 7, 5, 3), (5, 3, 12, 8, 64, 200))]


def _curves(seed):
    rng = np.random.default_rng(seed)
    return [synth.curve(rng, 3, 20, 333, knots="random", min_gap=0.01),
            synth.curve(rng, 2, 9, 50, knots="random", min_gap=0.01),
            synth.curve(rng, 4, 300, 2000, knots="uniform")]


def _oracle(kind, it, g):
    if kind == CURVE:
        return O.curve_vjp_homog(it.p, it.U, it.ctrl, it.u, g), O.curve_vjp(it.p, it.U, it.ctrl, it.u, g)[1]
    dpw = O.surface_vjp_homog(it.p, it.q, it.U, it.V, it.ctrl, it.u, it.v, g)
    _, dU, dV = O.surface_vjp(it.p, it.q, it.U, it.V, it.ctrl, it.u, it.v, g, want_ctrl=False)
    return dpw, (dU, dV)


@pytest.mark.parametrize("kind,warps,rows", [(SURF, 0, 0), (SURF, 2, 7), (SURF, 8, 32), (CURVE, 0, 0)])
def test_backward_homogeneous(kind, warps, rows):
    items = _surfaces(50) if kind == SURF else _curves(51)
    pk = pack(items, kind)
    plan = batch.Plan.for_packed(pk, warps=warps, rows=rows)
    plan.set_grad_homogeneous(True)
    kn, ct, pr = batch.to_device(pk)
    g = np.random.default_rng(8).normal(size=(pk.npts, 3)).astype(np.float32)
    gc, gk = torch.full_like(ct, float("nan")), torch.empty_like(kn)
    plan.backward(kn, ct, pr, torch.from_numpy(g).cuda(), gc, gk)
    assert plan.get_error()[0] == 0
    dcs = batch.unpack_ctrl(pk, gc.cpu().numpy())
    dks = batch.unpack_knots(pk, gk.cpu().numpy())
    for it, gi, dc, dk in zip(items, batch.unpack_points(pk, g), dcs, dks):
        ref, rk = _oracle(kind, it, gi)
        assert rel_inf(dc, ref) <= G_TOL
        if kind == SURF:       # knot gradients do not depend on the switch
            assert rel_inf(dk[0], rk[0]) <= G_TOL and rel_inf(dk[1], rk[1]) <= G_TOL
        else:
            assert rel_inf(dk, rk) <= G_TOL


def test_mse_and_fit_step_homogeneous():
    items = _surfaces(52)[:2]
    pk = pack(items, SURF)
    plan = batch.Plan.for_packed(pk)
    plan.set_grad_homogeneous(True)
    kn, ct, pr = batch.to_device(pk)
    T = np.random.default_rng(9).normal(size=(pk.npts, 3)).astype(np.float32)
    Td = torch.from_numpy(T).cuda()
    scale = 2.0 / (3.0 * pk.npts)
    gc = torch.empty_like(ct)
    plan.mse_fwd_bwd(kn, ct, pr, Td, None, gc, None, None, scale)
    dcs = batch.unpack_ctrl(pk, gc.cpu().numpy())
    grads = []
    for it, Ti, dc in zip(items, batch.unpack_points(pk, T), dcs):
        S = O.surface_eval(it.p, it.q, it.U, it.V, it.ctrl, it.u, it.v)
        gi = scale * (S - Ti)
        assert rel_inf(dc, O.surface_vjp_homog(it.p, it.q, it.U, it.V, it.ctrl, it.u, it.v, gi)) <= G_TOL
        grads.append(O.surface_vjp(it.p, it.q, it.U, it.V, it.ctrl, it.u, it.v, gi, want_knots=False)[0])
    # with the switch on, the fit step still updates (P, w) from the Cartesian gradient
    m, v = torch.zeros_like(ct), torch.zeros_like(ct)
    ct_fit = ct.clone()
    lr = 1e-3
    plan.fit_step(kn, ct_fit, pr, Td, m, v, 1, lr=lr, grad_scale=scale)
    after = batch.unpack_ctrl(pk, ct_fit.cpu().numpy())
    for it, dc, got in zip(items, grads, after):
        th, _, _ = O.adam(it.ctrl.astype(np.float64), dc, np.zeros_like(dc), np.zeros_like(dc), 1, lr=lr)
        sure = np.abs(dc) > 1e-2 * np.abs(dc).max()
        assert np.abs(got - th)[sure].max() <= 1e-3 * lr + 1e-6 * np.abs(th).max()
