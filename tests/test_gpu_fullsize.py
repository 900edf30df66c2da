"""Parity at the benchmark sizes, in the launch configurations the benchmark times,
against the FP64 oracle.

- The fused step on 256 bicubic 128x128 surfaces with the bench's tile (8 warps,
  128 rows): every item's points (element by element), loss, control-point and
  knot gradients.
- The 4096-curve fit workload: every curve's MSE gradients, and the Adam update
  wherever the gradient is not near zero.  At step 1, Adam's step is lr * sign(g),
  so a component whose gradient is near zero can flip under FP32 rounding.
- The 1000-surface ragged batch through the CUDA-graph engine, on a sample of
  items across all degree groups: points, loss and gradients."""
import numpy as np
import pytest
import torch

from gpu_util import G_TOL, S_TOL, bbox_diag, rel_inf
from oracle import oracle as O
from paper_2104_14547_gb300 import batch, engine, synth

pytestmark = pytest.mark.gpu


def _targets_gpu(pk, targets):
    tk = batch.pack_surfaces(targets) if pk.kind == 0 else batch.pack_curves(targets)
    kn, tct, pr = batch.to_device(tk)
    T = torch.empty((max(tk.npts, 1), 3), device="cuda")
    batch.Plan.for_packed(tk).eval(kn, tct, pr, T)
    return T


def test_bench_step_full_size():
    surfs, targets = synth.bicubic_batch(0, 256, 32, 128)
    pk = batch.pack_surfaces(surfs)
    kn, ct, pr = batch.to_device(pk)
    T = _targets_gpu(pk, targets)
    plan = batch.Plan.for_packed(pk, warps=8, rows=128)
    pts = torch.empty((pk.npts, 3), device="cuda")
    gc, gk = torch.empty_like(ct), torch.empty_like(kn)
    loss = torch.empty(pk.count, device="cuda")
    scale = 2.0 / (3.0 * pk.npts)
    plan.mse_fwd_bwd(kn, ct, pr, T, pts, gc, gk, loss, scale)
    assert plan.get_error()[0] == 0
    Tn = batch.unpack_points(pk, T.cpu().numpy())
    dcs = batch.unpack_ctrl(pk, gc.cpu().numpy())
    dks = batch.unpack_knots(pk, gk.cpu().numpy())
    lossn = loss.cpu().numpy()
    Sg = batch.unpack_points(pk, pts.cpu().numpy())
    worst = worst_s = 0.0
    for k, s in enumerate(surfs):
        S = O.surface_eval(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v)
        es = np.abs(Sg[k].astype(np.float64) - S).max() / bbox_diag(s.ctrl)
        worst_s = max(worst_s, es)
        assert es <= S_TOL, (k, es)
        Tk = Tn[k].astype(np.float64)
        g = scale * (S - Tk)
        dc, dU, dV = O.surface_vjp(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v, g)
        e = max(rel_inf(dcs[k], dc), rel_inf(dks[k][0], dU), rel_inf(dks[k][1], dV))
        worst = max(worst, e)
        assert e <= G_TOL, (k, e)
        ref_loss = float(((S - Tk) ** 2).sum())
        assert abs(lossn[k] - ref_loss) <= 1e-4 * ref_loss, (k, lossn[k], ref_loss)
    assert worst < G_TOL and worst_s <= S_TOL


def test_curve_fit_workload_full_size():
    curves, targets = synth.cubic_curve_batch(0, 4096, 64, 1024)
    pk = batch.pack_curves(curves)
    kn, ct, pr = batch.to_device(pk)
    T = _targets_gpu(pk, targets)
    plan = batch.Plan.for_packed(pk)
    scale = 2.0 / (3.0 * pk.npts)
    gc = torch.empty_like(ct)
    loss = torch.empty(pk.count, device="cuda")
    plan.mse_fwd_bwd(kn, ct, pr, T, None, gc, None, loss, scale)
    m, v = torch.zeros_like(ct), torch.zeros_like(ct)
    ct_fit = ct.clone()
    lr = 1e-3
    plan.fit_step(kn, ct_fit, pr, T, m, v, 1, lr=lr, grad_scale=scale)
    assert plan.get_error()[0] == 0
    Tn = batch.unpack_points(pk, T.cpu().numpy())
    dcs = batch.unpack_ctrl(pk, gc.cpu().numpy())
    after = batch.unpack_ctrl(pk, ct_fit.cpu().numpy())
    for k, c in enumerate(curves):
        S = O.curve_eval(c.p, c.U, c.ctrl, c.u)
        _, g = O.mse(S, Tn[k].astype(np.float64), 3 * pk.npts)
        dc, _ = O.curve_vjp(c.p, c.U, c.ctrl, c.u, g)
        assert rel_inf(dcs[k], dc) <= G_TOL, k
        th, _, _ = O.adam(c.ctrl.astype(np.float64), dc, np.zeros_like(dc), np.zeros_like(dc), 1, lr=lr)
        sure = np.abs(dc) > 1e-2 * np.abs(dc).max()
        assert np.abs(after[k] - th)[sure].max(initial=0.0) <= 1e-3 * lr + 1e-6 * np.abs(th).max()


def test_ragged_engine_full_size_sample():
    surfs, targets = synth.ragged_batch(0, 1000)
    pk = batch.pack_surfaces(surfs)
    T = _targets_gpu(pk, targets)
    eng = engine.RaggedEngine(surfs, T.cpu().numpy())
    eng.capture()
    eng.replay()
    torch.cuda.synchronize()
    assert all(e == 0 for e in eng.errors())
    Tn = batch.unpack_points(pk, T.cpu().numpy())
    dcs = batch.unpack_ctrl(pk, eng.grad_ctrl.cpu().numpy())
    dks = batch.unpack_knots(pk, eng.grad_knots.cpu().numpy())
    Sg = batch.unpack_points(pk, eng.pts.cpu().numpy())
    losses = eng.item_losses()
    rng = np.random.default_rng(0)
    sample = sorted(set(rng.choice(len(surfs), 24, replace=False).tolist()) | {0, len(surfs) - 1})
    for k in sample:
        s = surfs[k]
        S = O.surface_eval(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v)
        assert np.abs(Sg[k].astype(np.float64) - S).max() <= S_TOL * bbox_diag(s.ctrl), (k, "points")
        Tk = Tn[k].astype(np.float64)
        g = eng.grad_scale * (S - Tk)
        dc, dU, dV = O.surface_vjp(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v, g)
        assert rel_inf(dcs[k], dc) <= G_TOL, (k, "ctrl")
        assert rel_inf(dks[k][0], dU) <= G_TOL and rel_inf(dks[k][1], dV) <= G_TOL, (k, "knots")
        ref_loss = float(((S - Tk) ** 2).sum())
        assert abs(losses[k] - ref_loss) <= 1e-4 * ref_loss, k
