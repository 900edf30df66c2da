"""GPU parity: the libnurbs kernels (through the C-ABI) against the FP64 oracle on
the same seeded inputs.  Sizes span several tiles and ragged tails; edge cases
cover single samples, Bezier nets, repeated knots, samples on knots and empty
items."""
import numpy as np
import pytest
import torch

from gpu_util import G_TOL, check_points, gpu_eval, oracle_eval, oracle_vjp, pack, rel_inf
from oracle import oracle as O
from paper_2104_14547_gb300 import _lib, batch, synth

pytestmark = pytest.mark.gpu

SURF, CURVE = _lib.KIND_SURFACE, _lib.KIND_CURVE


def mixed_surfaces(seed, count=6):
    rng = np.random.default_rng(seed)
    out = []
    shapes = [(3, 3, 16, 16, 64, 64), (1, 2, 5, 7, 37, 300), (2, 5, 9, 12, 70, 41), (4, 1, 30, 6, 3, 129),
              (5, 4, 6, 5, 100, 33), (3, 3, 40, 33, 129, 257), (2, 2, 3, 3, 1, 1), (5, 5, 64, 64, 96, 96)]
    for k in range(count):
        p, q, n1, m1, nu, nv = shapes[k % len(shapes)]
        out.append(synth.surface(rng, p, q, n1, m1, nu, nv, knots="random" if k % 2 else "uniform",
                                 min_gap=1e-3))
    return out


def curves_mixed(seed):
    rng = np.random.default_rng(seed)
    # (degree, control points, samples): the curve kernels take up to 256 control
    # points, longer polygons go to the tile kernels; (2, 60, 4) jumps over spans
    specs = [(3, 64, 1024), (1, 2, 5), (2, 17, 300), (4, 9, 33), (5, 6, 1), (3, 100, 2049), (2, 3, 257),
             (3, 300, 700), (2, 60, 4), (5, 256, 3001), (1, 40, 129)]
    # every knot gap >= 1e-3 is out of reach for hundreds of knots: scale the gap
    return [synth.curve(rng, p, n1, nu, min_gap=min(1e-3, 0.01 / n1)) for p, n1, nu in specs]


# ------------------------------------------------------------------- forward
def test_forward_single_bicubic_uniform():
    s = synth.single_bicubic(0)
    _, got = gpu_eval([s], SURF)
    check_points([s], SURF, got)


def test_forward_mixed_degrees_ragged():
    surfs = mixed_surfaces(1, 8)
    _, got = gpu_eval(surfs, SURF)
    check_points(surfs, SURF, got)


@pytest.mark.parametrize("warps,rows", [(1, 0), (2, 5), (4, 0), (4, 3), (4, 64), (8, 0), (8, 128), (8, 9)])
def test_forward_tile_shapes(warps, rows):
    surfs = mixed_surfaces(2, 6)
    _, got = gpu_eval(surfs, SURF, warps=warps, rows=rows)
    check_points(surfs, SURF, got)


def test_forward_curves():
    cs = curves_mixed(3)
    _, got = gpu_eval(cs, CURVE)
    check_points(cs, CURVE, got)


def test_curves_clustered_samples():
    # samples in two clusters far apart in span: within one warp step some lanes are
    # past the 32 staged knots of the forward's span search and take its fallback
    # while the others do not; the gradient kernels' lanes jump many spans at once
    rng = np.random.default_rng(44)
    items = []
    for p, n1 in ((3, 200), (2, 256), (5, 90)):
        c = synth.curve(rng, p, n1, 2, knots="uniform")
        u = np.concatenate([np.linspace(0.0, 0.02, 20), np.linspace(0.97, 1.0, 23)]).astype(np.float32)
        items.append(synth.Curve(p, c.U, c.ctrl, np.sort(u)))
        u2 = np.concatenate([np.linspace(0.0, 0.3, 7), np.linspace(0.31, 0.32, 70),
                             np.linspace(0.6, 1.0, 9)]).astype(np.float32)
        items.append(synth.Curve(p, c.U, c.ctrl, np.sort(u2)))
    _, got = gpu_eval(items, CURVE)
    check_points(items, CURVE, got)
    pk, g, gc, gk = _run_backward(items, CURVE, 44)
    _check_grads(items, CURVE, pk, g, gc, gk)


def test_forward_curve_edge_cases():
    # small curves (a small shared layout per warp) of every degree
    rng = np.random.default_rng(46)
    items = []
    for p in (1, 2, 3, 4, 5):
        c = synth.curve(rng, p, 20, 2, knots="uniform")
        U = c.U.copy()
        U[p + 3:2 * p + 3] = U[p + 3]   # an interior knot of multiplicity p: spans of zero length
        u = np.sort(np.concatenate([np.linspace(0.0, 1.0, 61), U[p:20 + 1]]).astype(np.float32))   # samples on every knot
        items.append(synth.Curve(p, U, c.ctrl, u))
        # clustered samples: some lanes of a warp step pass the 32 staged knots
        c2 = synth.curve(rng, p, 60, 2, knots="uniform")
        u2 = np.concatenate([np.linspace(0.0, 0.02, 20), np.linspace(0.97, 1.0, 23)]).astype(np.float32)
        items.append(synth.Curve(p, c2.U, c2.ctrl, np.sort(u2)))
    # a single Bezier span (n = p), a one-sample curve and an empty one
    items.append(synth.Curve(3, np.array([0, 0, 0, 0, 1, 1, 1, 1], np.float32),
                             synth.random_walk_polygon(rng, 4), synth.uniform_params(33)))
    items.append(synth.curve(rng, 2, 7, 1))
    items.append(synth.curve(rng, 3, 12, 0))
    _, got = gpu_eval(items, CURVE)
    check_points(items, CURVE, got)
    # clamped knots interpolate the end points
    c = synth.Curve(3, synth.clamped_uniform_knots(10, 3), synth.random_walk_polygon(rng, 10),
                    np.array([0.0, 1.0], np.float32))
    _, g = gpu_eval([c], CURVE)
    np.testing.assert_allclose(g[0][0], c.ctrl[0, :3], atol=1e-6)
    np.testing.assert_allclose(g[0][1], c.ctrl[-1, :3], atol=1e-6)


def test_forward_edge_cases():
    rng = np.random.default_rng(4)
    # Bezier nets (n = p), samples exactly on uniform knots, a double interior knot,
    # single-sample grids and an empty item
    bez = synth.Surface(3, 2, np.array([0, 0, 0, 0, 1, 1, 1, 1], np.float32), np.array([0, 0, 0, 1, 1, 1], np.float32),
                        synth.planar_net(rng, 4, 3), synth.uniform_params(17), synth.uniform_params(9))
    onk = synth.surface(rng, 3, 3, 16, 16, 14, 27, knots="uniform")           # u = a/13 hits every knot
    rep = synth.surface(rng, 2, 3, 8, 9, 50, 60)
    rep.U = rep.U.copy()
    rep.U[4] = rep.U[5]
    one = synth.surface(rng, 2, 2, 5, 5, 1, 1)
    empty = synth.surface(rng, 3, 3, 6, 6, 0, 10)
    items = [bez, onk, rep, one, empty]
    pk, got = gpu_eval(items, SURF)
    check_points(items, SURF, got)
    # endpoint interpolation on clamped knots survives FP32
    c = synth.surface(rng, 3, 3, 10, 10, 2, 2)
    _, g = gpu_eval([c], SURF)
    np.testing.assert_allclose(g[0][0, 0], c.ctrl[0, 0, :3], atol=1e-6)
    np.testing.assert_allclose(g[0][1, 1], c.ctrl[-1, -1, :3], atol=1e-6)


def test_rational_circle_gpu():
    import json
    import os
    gl = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "rational_circle.json")))
    c = gl["full_circle"]
    cur = synth.Curve(c["p"], np.array(c["U"], np.float32), np.array(c["ctrl"], np.float32), synth.uniform_params(1001))
    _, got = gpu_eval([cur], CURVE)
    r = np.linalg.norm(got[0].astype(np.float64), axis=1)
    assert np.abs(r - 1).max() < 1e-6


# ------------------------------------------------------------------ backward
def _run_backward(items, kind, seed, knots=True, **plan_kw):
    pk = pack(items, kind)
    plan = batch.Plan.for_packed(pk, **plan_kw)
    kn, ct, pr = batch.to_device(pk)
    rng = np.random.default_rng(seed)
    g = rng.normal(size=(max(pk.npts, 1), 3)).astype(np.float32)
    gd = torch.from_numpy(g).cuda()
    gctrl = torch.full_like(ct, float("nan"))
    gkn = torch.full_like(kn, float("nan")) if knots else None
    plan.backward(kn, ct, pr, gd, gctrl, gkn)
    st, flags = plan.get_error()
    assert st == 0, (st, flags)
    return pk, g, gctrl.cpu().numpy(), (gkn.cpu().numpy() if knots else None)


def _check_grads(items, kind, pk, g, gctrl, gkn):
    gs = batch.unpack_points(pk, g)
    dcs = batch.unpack_ctrl(pk, gctrl)
    dks = batch.unpack_knots(pk, gkn) if gkn is not None else [None] * len(items)
    worst = 0.0
    for it, gi, dc, dk in zip(items, gs, dcs, dks):
        rc, rU, rV = oracle_vjp(it, kind, gi)
        e = rel_inf(dc, rc)
        worst = max(worst, e)
        assert e <= G_TOL, ("ctrl", e)
        if dk is not None:
            if kind == CURVE:
                e = rel_inf(dk, rU)
                assert e <= G_TOL, ("U", e)
            else:
                e1, e2 = rel_inf(dk[0], rU), rel_inf(dk[1], rV)
                assert e1 <= G_TOL and e2 <= G_TOL, ("UV", e1, e2)
                e = max(e1, e2)
            worst = max(worst, e)
    return worst


def test_backward_surfaces_mixed():
    items = mixed_surfaces(5, 8)
    pk, g, gc, gk = _run_backward(items, SURF, 5)
    _check_grads(items, SURF, pk, g, gc, gk)


def test_backward_without_knots_matches():
    items = mixed_surfaces(6, 5)
    pk, g, gc, _ = _run_backward(items, SURF, 6, knots=False)
    _check_grads(items, SURF, pk, g, gc, None)


@pytest.mark.parametrize("warps,rows", [(1, 0), (2, 7), (4, 2), (4, 100), (8, 0), (8, 64), (8, 200), (6, 50)])
def test_backward_tile_shapes(warps, rows):
    items = mixed_surfaces(7, 6)
    pk, g, gc, gk = _run_backward(items, SURF, 7, warps=warps, rows=rows)
    _check_grads(items, SURF, pk, g, gc, gk)


def test_backward_curves_repeated_knots():
    rng = np.random.default_rng(18)
    items = []
    for p, n1, nu in ((3, 12, 400), (2, 300, 900)):         # curve kernels, then the tile kernels
        c = synth.curve(rng, p, n1, nu, knots="uniform")
        U = c.U.copy()
        U[p + 3] = U[p + 4]                                 # a double interior knot
        items.append(synth.Curve(p, U, c.ctrl, c.u))
    pk, g, gc, gk = _run_backward(items, CURVE, 18)
    _check_grads(items, CURVE, pk, g, gc, gk)


def test_backward_curves():
    items = curves_mixed(8)
    pk, g, gc, gk = _run_backward(items, CURVE, 8)
    _check_grads(items, CURVE, pk, g, gc, gk)


def test_backward_edge_cases():
    rng = np.random.default_rng(9)
    onk = synth.surface(rng, 3, 3, 16, 16, 14, 27, knots="uniform")
    one = synth.surface(rng, 2, 2, 5, 5, 1, 1)
    empty = synth.surface(rng, 3, 3, 6, 6, 0, 10)
    sparse = synth.surface(rng, 3, 2, 40, 30, 5, 4)       # samples jump over many spans
    rep = synth.surface(rng, 2, 3, 8, 9, 50, 60)          # repeated interior knots: 0/0 := 0 in Eq. 4
    rep.U = rep.U.copy()
    rep.U[4] = rep.U[5]                                   # a double knot in u
    rep.V = rep.V.copy()
    rep.V[5] = rep.V[6] = rep.V[7]                        # a triple knot in v (C0 across it)
    items = [onk, one, empty, sparse, rep]
    pk, g, gc, gk = _run_backward(items, SURF, 9)
    # sample-on-knot items: control/weight gradients are exact, knot gradients one-sided
    _check_grads(items, SURF, pk, g, gc, gk)
    dc = batch.unpack_ctrl(pk, gc)
    assert np.all(dc[2] == 0)                            # no samples -> zero gradient


def test_determinism_and_batch_invariance():
    items = mixed_surfaces(10, 6)
    r1 = _run_backward(items, SURF, 10)
    r2 = _run_backward(items, SURF, 10)
    assert np.array_equal(r1[2], r2[2]) and np.array_equal(r1[3], r2[3])
    # item 3 alone gives the same bits as inside the batch
    pk, g, gc, gk = r1
    alone = _run_backward([items[3]], SURF, 10)
    g3 = batch.unpack_points(pk, g)[3]
    pk1 = pack([items[3]], SURF)
    plan = batch.Plan.for_packed(pk1)
    kn, ct, pr = batch.to_device(pk1)
    gctrl = torch.zeros_like(ct)
    gkn = torch.zeros_like(kn)
    plan.backward(kn, ct, pr, torch.from_numpy(np.ascontiguousarray(g3.reshape(-1, 3))).cuda(), gctrl, gkn)
    assert np.array_equal(batch.unpack_ctrl(pk1, gctrl.cpu().numpy())[0], batch.unpack_ctrl(pk, gc)[3])
    del alone


# --------------------------------------------------------------- fused MSE
def _targets_oracle(items, targets, kind):
    return [oracle_eval(t, kind).astype(np.float32) for t in targets]


def test_mse_fwd_bwd_matches_oracle_chain():
    surfs, tg = synth.bicubic_batch(11, batch=5, net=12, grid=45)
    T = _targets_oracle(surfs, tg, SURF)
    pk = pack(surfs, SURF)
    plan = batch.Plan.for_packed(pk)
    kn, ct, pr = batch.to_device(pk)
    Td = torch.from_numpy(np.concatenate([t.reshape(-1, 3) for t in T])).cuda()
    pts = torch.zeros((pk.npts, 3), device="cuda")
    gc = torch.zeros_like(ct)
    gk = torch.zeros_like(kn)
    loss = torch.zeros(len(surfs), device="cuda")
    scale = 2.0 / (3 * pk.npts)
    plan.mse_fwd_bwd(kn, ct, pr, Td, pts, gc, gk, loss, scale)
    assert plan.get_error()[0] == 0
    check_points(surfs, SURF, batch.unpack_points(pk, pts.cpu().numpy()))
    Ls = []
    for k, (s, t) in enumerate(zip(surfs, T)):
        S = oracle_eval(s, SURF)
        L, gref = O.mse(S, t.astype(np.float64), 3 * pk.npts)
        Ls.append(L * 3 * pk.npts)
        rc, rU, rV = oracle_vjp(s, SURF, gref)
        assert rel_inf(batch.unpack_ctrl(pk, gc.cpu().numpy())[k], rc) <= G_TOL
        dU, dV = batch.unpack_knots(pk, gk.cpu().numpy())[k]
        assert rel_inf(dU, rU) <= G_TOL and rel_inf(dV, rV) <= G_TOL
    np.testing.assert_allclose(loss.cpu().numpy(), Ls, rtol=1e-4)


def test_fit_step_one_adam_step_curves():
    curves, tg = synth.cubic_curve_batch(12, batch=7, n1=20, samples=300)
    T = _targets_oracle(curves, tg, CURVE)
    pk = pack(curves, CURVE)
    plan = batch.Plan.for_packed(pk)
    kn, ct, pr = batch.to_device(pk)
    Td = torch.from_numpy(np.concatenate(T)).cuda()
    m = torch.zeros_like(ct)
    v = torch.zeros_like(ct)
    loss = torch.zeros(len(curves), device="cuda")
    lr = 1e-2
    for step in (1, 2):
        c_before = batch.unpack_ctrl(pk, ct.cpu().numpy())
        m_before, v_before = m.cpu().numpy().copy(), v.cpu().numpy().copy()
        plan.fit_step(kn, ct, pr, Td, m, v, step, lr=lr, loss_items=loss)
        assert plan.get_error()[0] == 0
        after = batch.unpack_ctrl(pk, ct.cpu().numpy())
        for k, c in enumerate(curves):
            cb = c_before[k].astype(np.float64)
            S = O.curve_eval(c.p, c.U, cb, c.u)
            _, g = O.mse(S, T[k].astype(np.float64), 3 * pk.npts)
            dc, _ = O.curve_vjp(c.p, c.U, cb, c.u, g)
            mb = batch.unpack_ctrl(pk, m_before)[k]
            vb = batch.unpack_ctrl(pk, v_before)[k]
            th, _, _ = O.adam(cb, dc, mb, vb, step, lr=lr)
            # the Adam step is lr-sized, so compare it relative to lr
            assert np.abs(after[k] - th).max() <= 1e-3 * lr + 1e-6 * np.abs(th).max()


def test_fit_step_surfaces_and_loss_decreases():
    surfs, tg = synth.bicubic_batch(13, batch=4, net=10, grid=40)
    T = _targets_oracle(surfs, tg, SURF)
    pk = pack(surfs, SURF)
    plan = batch.Plan.for_packed(pk)
    kn, ct, pr = batch.to_device(pk)
    Td = torch.from_numpy(np.concatenate([t.reshape(-1, 3) for t in T])).cuda()
    m, v = torch.zeros_like(ct), torch.zeros_like(ct)
    loss = torch.zeros(len(surfs), device="cuda")
    hist = []
    for step in range(1, 31):
        plan.fit_step(kn, ct, pr, Td, m, v, step, lr=1e-2, loss_items=loss)
        hist.append(loss.sum().item())
    assert hist[-1] < 0.5 * hist[0]


def _fit_once_against_oracle(items, kind, lr=1e-2):
    rng = np.random.default_rng(45)
    pk = pack(items, kind)
    T = rng.normal(size=(max(pk.npts, 1), 3)).astype(np.float32)
    plan = batch.Plan.for_packed(pk)
    kn, ct, pr = batch.to_device(pk)
    m, v = torch.zeros_like(ct), torch.zeros_like(ct)
    loss = torch.full((pk.count,), float("nan"), device="cuda")
    before = batch.unpack_ctrl(pk, ct.cpu().numpy())
    plan.fit_step(kn, ct, pr, torch.from_numpy(T).cuda(), m, v, 1, lr=lr, loss_items=loss)
    assert plan.get_error()[0] == 0
    after = batch.unpack_ctrl(pk, ct.cpu().numpy())
    mm = batch.unpack_ctrl(pk, m.cpu().numpy())
    lossn = loss.cpu().numpy()
    for k, (it, Tk) in enumerate(zip(items, batch.unpack_points(pk, T))):
        c0 = before[k].astype(np.float64)
        npts = Tk.reshape(-1, 3).shape[0]
        if npts == 0:                       # no samples: zero gradient, no move, zero loss
            assert np.array_equal(after[k], before[k]) and np.all(mm[k] == 0) and lossn[k] == 0
            continue
        if kind == CURVE:
            S = O.curve_eval(it.p, it.U, c0, it.u)
            _, g = O.mse(S, Tk.astype(np.float64), 3 * pk.npts)
            dc, _ = O.curve_vjp(it.p, it.U, c0, it.u, g, want_knots=False)
        else:
            S = O.surface_eval(it.p, it.q, it.U, it.V, c0, it.u, it.v)
            _, g = O.mse(S, Tk.astype(np.float64), 3 * pk.npts)
            dc, _, _ = O.surface_vjp(it.p, it.q, it.U, it.V, c0, it.u, it.v, g, want_knots=False)
        th, _, _ = O.adam(c0, dc, np.zeros_like(dc), np.zeros_like(dc), 1, lr=lr)
        sure = np.abs(dc) > 1e-2 * np.abs(dc).max()
        assert np.abs(after[k] - th)[sure].max(initial=0.0) <= 1e-3 * lr + 1e-6 * np.abs(th).max(), k
        assert abs(lossn[k] - float(((S - Tk) ** 2).sum())) <= 1e-4 * float(((S - Tk) ** 2).sum()) + 1e-6


def test_fit_step_empty_and_single_sample_items():
    rng = np.random.default_rng(46)
    surfs = [synth.surface(rng, 3, 3, 8, 8, 20, 20), synth.surface(rng, 3, 3, 6, 6, 0, 10),
             synth.surface(rng, 2, 3, 7, 6, 12, 0), synth.surface(rng, 3, 3, 9, 7, 1, 1),
             synth.surface(rng, 3, 3, 10, 10, 33, 17)]
    _fit_once_against_oracle(surfs, SURF)
    curves = [synth.curve(rng, 3, 20, 200), synth.curve(rng, 3, 12, 0), synth.curve(rng, 2, 9, 1),
              synth.curve(rng, 4, 300, 0, knots="uniform"), synth.curve(rng, 4, 300, 500, knots="uniform"), synth.curve(rng, 5, 64, 37)]
    _fit_once_against_oracle(curves, CURVE)


# ------------------------------------------------------------- device checks
def test_device_checks_flag_bad_inputs():
    rng = np.random.default_rng(14)
    s = synth.surface(rng, 3, 3, 8, 8, 20, 20)
    bad_knots = synth.Surface(s.p, s.q, s.U[::-1].copy(), s.V, s.ctrl, s.u, s.v)
    _check_flag([bad_knots], 2)
    out = synth.Surface(s.p, s.q, s.U, s.V, s.ctrl, s.u * 1.5, s.v)
    _check_flag([out], 4)
    unsorted = synth.Surface(s.p, s.q, s.U, s.V, s.ctrl, s.u[::-1].copy(), s.v)
    _check_flag([unsorted], 5)


def test_device_checks_flag_bad_curves():
    rng = np.random.default_rng(15)
    for n1, nu in ((20, 300), (300, 500)):          # curve kernels, then the tile kernels
        c = synth.curve(rng, 3, n1, nu, min_gap=1e-5)
        _check_flag([synth.Curve(c.p, c.U[::-1].copy(), c.ctrl, c.u)], 2, CURVE)
        _check_flag([synth.Curve(c.p, c.U, c.ctrl, c.u * 1.5)], 4, CURVE)
        _check_flag([synth.Curve(c.p, c.U, c.ctrl, c.u[::-1].copy())], 5, CURVE)


def _check_flag(items, status, kind=None):
    kind = SURF if kind is None else kind
    pk = pack(items, kind)
    plan = batch.Plan.for_packed(pk)
    kn, ct, pr = batch.to_device(pk)
    pts = torch.zeros((pk.npts, 3), device="cuda")
    plan.eval(kn, ct, pr, pts)
    st, flags = plan.get_error()
    assert flags & (1 << status), (st, flags)
    gc = torch.zeros_like(ct)
    plan.backward(kn, ct, pr, torch.zeros_like(pts), gc, torch.zeros_like(kn))
    st, flags = plan.get_error()
    assert flags & (1 << status), (st, flags)
    # the workspace stays usable: a clean call afterwards reports nothing
    assert plan.get_error()[0] == 0


def test_item_mean_loss_scale_matches_oracle():
    # each item's own MSE normalisation (descriptor grad_scale = 2 / (3 x its points)):
    # the call's grad_scale is ignored and every gradient matches the oracle's for that
    # item's own mean, on the curve kernels, the tile path for long curves and surfaces
    rng = np.random.default_rng(53)
    curves = [synth.curve(rng, 3, 20, 300), synth.curve(rng, 4, 300, 700, knots="uniform"), synth.curve(rng, 2, 12, 50)]
    surfs = [synth.surface(rng, 3, 3, 10, 10, 40, 30), synth.surface(rng, 2, 4, 8, 9, 25, 70)]
    for items, kind in ((curves, CURVE), (surfs, SURF)):
        pk = pack(items, kind)
        plan = batch.Plan.for_packed(pk, item_mean=True)
        kn, ct, pr = batch.to_device(pk)
        T = rng.normal(size=(pk.npts, 3)).astype(np.float32)
        gc = torch.zeros_like(ct)
        loss = torch.zeros(pk.count, device="cuda")
        plan.mse_fwd_bwd(kn, ct, pr, torch.from_numpy(T).cuda(), None, gc, None, loss, grad_scale=123.0)
        assert plan.get_error()[0] == 0
        dcs = batch.unpack_ctrl(pk, gc.cpu().numpy())
        for k, (it, Tk) in enumerate(zip(items, batch.unpack_points(pk, T))):
            S = oracle_eval(it, kind)
            Tk = Tk.reshape(S.shape).astype(np.float64)
            _, g = O.mse(S, Tk, 3 * Tk.reshape(-1, 3).shape[0])
            dc = oracle_vjp(it, kind, g)[0]
            assert rel_inf(dcs[k], dc) <= G_TOL, (kind, k)
