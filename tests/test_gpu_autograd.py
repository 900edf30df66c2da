"""The torch.autograd layers: forward against the oracle, gradients through
loss.backward() against the oracle's vector-Jacobian product, and a short fit."""
import numpy as np
import pytest
import torch

from gpu_util import G_TOL, S_TOL, bbox_diag, rel_inf
from oracle import oracle as O
from paper_2104_14547_gb300 import autograd as A
from paper_2104_14547_gb300 import batch, synth

pytestmark = pytest.mark.gpu


def test_surface_layer_forward_backward_vs_oracle():
    rng = np.random.default_rng(31)
    surfs = [synth.surface(rng, 3, 2, 9, 8, 40, 33), synth.surface(rng, 2, 3, 12, 14, 17, 70)]
    layer = A.NurbsSurface(surfs, learn_knots=True)
    pts = layer()
    g = torch.randn_like(pts)
    (pts * g).sum().backward()
    per = layer.split(pts.detach())
    gs = layer.split(g)
    dc = batch.unpack_ctrl(layer.packed, layer.ctrl.grad.cpu().numpy())
    dk = batch.unpack_knots(layer.packed, layer.knots.grad.cpu().numpy())
    for k, s in enumerate(surfs):
        ref = O.surface_eval(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v)
        assert np.abs(per[k].cpu().numpy() - ref).max() <= S_TOL * bbox_diag(s.ctrl)
        rc, rU, rV = O.surface_vjp(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v, gs[k].cpu().numpy())
        assert rel_inf(dc[k], rc) <= G_TOL
        assert rel_inf(dk[k][0], rU) <= G_TOL and rel_inf(dk[k][1], rV) <= G_TOL


def test_curve_layer_and_bspline_weights_fixed():
    rng = np.random.default_rng(32)
    curves = [synth.curve(rng, 3, 20, 200), synth.curve(rng, 2, 9, 77)]
    layer = A.BSplineCurve(curves)
    assert not hasattr(layer, "ctrl") and layer.weights.requires_grad is False
    pts = layer()
    g = torch.randn_like(pts)
    (pts * g).sum().backward()
    dxyz = layer.xyz.grad.cpu().numpy()
    off = 0
    for k, c in enumerate(curves):
        c1 = c.ctrl.copy()
        c1[:, 3] = 1.0
        rc, _ = O.curve_vjp(c.p, c.U, c1, c.u, g[off: off + len(c.u)].cpu().numpy())
        assert rel_inf(dxyz[int(layer.packed.descs[k]["ctrl"]): int(layer.packed.descs[k]["ctrl"]) + c.n1], rc[:, :3]) <= G_TOL
        off += len(c.u)


def test_fit_with_torch_adam_reduces_loss():
    surfs, tg = synth.bicubic_batch(33, batch=3, net=10, grid=40)
    T = torch.from_numpy(np.concatenate([O.surface_eval(t.p, t.q, t.U, t.V, t.ctrl, t.u, t.v).reshape(-1, 3)
                                         for t in tg]).astype(np.float32)).cuda()
    layer = A.NurbsSurface(surfs)
    opt = torch.optim.Adam(layer.parameters(), lr=1e-2)
    losses = []
    for _ in range(40):
        opt.zero_grad()
        loss = torch.nn.functional.mse_loss(layer(), T)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert losses[-1] < 0.5 * losses[0]
