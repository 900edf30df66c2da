"""GPU knot gradients with the paper's Gaussian-smoothed indicator (Sec. 3.2,
nurbs_plan_set_knot_sigma) against the FP64 oracle.

Samples are placed within a fraction of sigma of interior knots, where the
smoothed term matters.  The test first checks that the oracle's gradient with
sigma differs from the sigma -> 0 one, and checks the GPU against that
difference as well as against the whole gradient.  The
paths covered: surface tiles (single- and multi-tile), the fused MSE step,
curves on the curve kernels and on the tile kernels."""
import numpy as np
import pytest
import torch

from gpu_util import G_TOL, pack
from oracle import oracle as O
from paper_2104_14547_gb300 import _lib, batch, synth

pytestmark = pytest.mark.gpu
SURF, CURVE = _lib.KIND_SURFACE, _lib.KIND_CURVE
GAP = 0.02
SIGMA = GAP / 8


def _near_knot_params(U, p, n_uniform, rng):
    inner = U[p + 1: len(U) - p - 1].astype(np.float64)
    extra = [k + f * SIGMA for k in inner for f in (-0.6, -0.2, 0.25, 0.7)]
    u = np.concatenate([np.linspace(0.0, 1.0, n_uniform), extra, rng.uniform(0, 1, 5)])
    return np.unique(np.clip(u, 0.0, 1.0).astype(np.float32))


def _surfaces(seed):
    rng = np.random.default_rng(seed)
    out = []
    for p, q, n1, m1 in ((3, 3, 10, 9), (2, 4, 8, 11), (1, 2, 6, 7), (5, 3, 12, 8)):
        s = synth.surface(rng, p, q, n1, m1, 4, 4, knots="random", min_gap=GAP)
        out.append(synth.Surface(p, q, s.U, s.V, s.ctrl, _near_knot_params(s.U, p, 30, rng),
                                 _near_knot_params(s.V, q, 25, rng)))
    return out


def _run(items, kind, **plan_kw):
    pk = pack(items, kind)
    plan = batch.Plan.for_packed(pk, **plan_kw)
    plan.set_knot_sigma(SIGMA)
    kn, ct, pr = batch.to_device(pk)
    rng = np.random.default_rng(7)
    g = rng.normal(size=(max(pk.npts, 1), 3)).astype(np.float32)
    gc, gk = torch.empty_like(ct), torch.full_like(kn, float("nan"))
    plan.backward(kn, ct, pr, torch.from_numpy(g).cuda(), gc, gk)
    assert plan.get_error()[0] == 0
    return pk, g, batch.unpack_knots(pk, gk.cpu().numpy())


def _close(got, ref, ref0, require_part=True):
    """The GPU reproduces the smoothed term: its error is small against the
    gradient and against the term itself (ref - ref0), which must not vanish
    (when required: the backward cases are built so that it does not)."""
    part = np.abs(ref - ref0).max()
    scale = np.abs(ref).max()
    if require_part:
        assert part > 1e-4 * scale, (part, scale)
    err = np.abs(got - ref).max()
    assert err <= G_TOL * scale, err / scale
    assert err <= 0.05 * part + 2e-5 * scale, (err, part)


def _check(items, kind, pk, g, dks):
    gs = batch.unpack_points(pk, g)
    for it, gi, dk in zip(items, gs, dks):
        if kind == CURVE:
            _, rU = O.curve_vjp(it.p, it.U, it.ctrl, it.u, gi, knot_sigma=SIGMA)
            _, r0 = O.curve_vjp(it.p, it.U, it.ctrl, it.u, gi)
            _close(dk, rU, r0)
        else:
            _, rU, rV = O.surface_vjp(it.p, it.q, it.U, it.V, it.ctrl, it.u, it.v, gi, knot_sigma=SIGMA)
            _, r0U, r0V = O.surface_vjp(it.p, it.q, it.U, it.V, it.ctrl, it.u, it.v, gi)
            _close(dk[0], rU, r0U)
            _close(dk[1], rV, r0V)


@pytest.mark.parametrize("warps,rows", [(0, 0), (2, 7), (8, 32)])
def test_sigma_knot_gradients_surfaces(warps, rows):
    items = _surfaces(31)
    pk, g, dks = _run(items, SURF, warps=warps, rows=rows)
    _check(items, SURF, pk, g, dks)


def test_sigma_knot_gradients_fused_mse():
    items = _surfaces(32)[:2]
    pk = pack(items, SURF)
    plan = batch.Plan.for_packed(pk)
    plan.set_knot_sigma(SIGMA)
    kn, ct, pr = batch.to_device(pk)
    rng = np.random.default_rng(9)
    T = rng.normal(size=(pk.npts, 3)).astype(np.float32)
    gc, gk = torch.empty_like(ct), torch.empty_like(kn)
    loss = torch.zeros(pk.count, device="cuda")
    scale = 2.0 / (3.0 * pk.npts)
    plan.mse_fwd_bwd(kn, ct, pr, torch.from_numpy(T).cuda(), None, gc, gk, loss, scale)
    dks = batch.unpack_knots(pk, gk.cpu().numpy())
    for it, Ti, dk in zip(items, batch.unpack_points(pk, T), dks):
        S = O.surface_eval(it.p, it.q, it.U, it.V, it.ctrl, it.u, it.v)
        gi = scale * (S - Ti)
        _, rU, rV = O.surface_vjp(it.p, it.q, it.U, it.V, it.ctrl, it.u, it.v, gi, knot_sigma=SIGMA)
        _, r0U, r0V = O.surface_vjp(it.p, it.q, it.U, it.V, it.ctrl, it.u, it.v, gi)
        _close(dk[0], rU, r0U, require_part=False)
        _close(dk[1], rV, r0V, require_part=False)


def test_sigma_knot_gradients_curves():
    rng = np.random.default_rng(33)
    items = []
    # curve kernels (random knots), then the tile kernels (300 points, uniform knots:
    # random knots that far apart in count cannot all keep a gap of a few sigma)
    for p, n1, kn in ((3, 20, "random"), (2, 9, "random"), (4, 300, "uniform")):
        c = synth.curve(rng, p, n1, 4, knots=kn, min_gap=GAP)
        items.append(synth.Curve(p, c.U, c.ctrl, _near_knot_params(c.U, p, 200, rng)))
    pk, g, dks = _run(items, CURVE)
    _check(items, CURVE, pk, g, dks)


def test_sigma_zero_is_the_default_reading():
    items = _surfaces(34)[:2]
    pk = pack(items, SURF)
    plan = batch.Plan.for_packed(pk)
    kn, ct, pr = batch.to_device(pk)
    g = torch.randn((pk.npts, 3), device="cuda")
    gk0, gk1 = torch.empty_like(kn), torch.empty_like(kn)
    gc = torch.empty_like(ct)
    plan.backward(kn, ct, pr, g, gc, gk0)
    plan.set_knot_sigma(SIGMA)
    plan.set_knot_sigma(0.0)
    plan.backward(kn, ct, pr, g, gc, gk1)
    assert torch.equal(gk0, gk1)
