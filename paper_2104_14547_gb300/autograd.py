"""PyTorch layers over libnurbs (the module form the paper describes in Sec. 3.3
and its implementation appendix): a torch.autograd.Function whose forward calls
nurbs_eval_surface / nurbs_eval_curve and whose backward calls nurbs_backward,
recomputing the basis instead of storing it.

NurbsSurface / NurbsCurve hold a packed batch with learnable control points and
weights (and, optionally, knots).  BSplineSurface / BSplineCurve fix every weight
to 1 (the paper's B-spline layer); their control points are the only parameters
unless knots are learned too (the paper's NUBS case).
"""
from __future__ import annotations

import numpy as np
import torch
from torch import nn

from . import _lib, batch


class NurbsEvalFunction(torch.autograd.Function):
    """pts = S(ctrl, knots) for a packed batch; params (the samples) are constant."""

    @staticmethod
    def forward(ctx, ctrl, knots, params, plan):
        ctrl = ctrl.contiguous()
        knots = knots.contiguous()
        pts = torch.empty((max(plan.points, 1), 3), device=ctrl.device, dtype=torch.float32)
        plan.eval(knots, ctrl, params, pts)
        ctx.save_for_backward(ctrl, knots, params)
        ctx.plan = plan
        return pts[: plan.points]

    @staticmethod
    def backward(ctx, grad_pts):
        ctrl, knots, params = ctx.saved_tensors
        plan = ctx.plan
        gc = torch.empty_like(ctrl) if ctx.needs_input_grad[0] else None
        gk = torch.empty_like(knots) if ctx.needs_input_grad[1] else None
        if gc is None and gk is None:
            return None, None, None, None
        g = grad_pts.contiguous()
        if g.shape[0] == 0:
            g = torch.zeros((1, 3), device=ctrl.device)
        plan.backward(knots, ctrl, params, g, gc, gk)
        return gc, gk, None, None


def nurbs_eval(ctrl, knots, params, plan):
    return NurbsEvalFunction.apply(ctrl, knots, params, plan)


class _Layer(nn.Module):
    def __init__(self, packed: batch.Packed, learn_knots: bool, learn_weights: bool, device, **plan_kw):
        super().__init__()
        self.packed = packed
        self.plan = batch.Plan.for_packed(packed, device=device, **plan_kw)
        kn, ct, pr = batch.to_device(packed, device)
        self.learn_weights = learn_weights
        if learn_weights:
            self.ctrl = nn.Parameter(ct)
        else:
            self.xyz = nn.Parameter(ct[:, :3].contiguous())
            self.register_buffer("weights", torch.ones_like(ct[:, 3:]))
        if learn_knots:
            self.knots = nn.Parameter(kn)
        else:
            self.register_buffer("knots", kn)
        self.register_buffer("params", pr)

    def control_net(self) -> torch.Tensor:
        """(x, y, z, w) per control point in the packed layout."""
        if self.learn_weights:
            return self.ctrl
        return torch.cat([self.xyz, self.weights], dim=1)

    def forward(self) -> torch.Tensor:
        """Evaluated points, [total points, 3] in the packed layout."""
        return nurbs_eval(self.control_net(), self.knots, self.params, self.plan)

    def split(self, pts: torch.Tensor):
        """Per-item views of a packed point tensor."""
        out = []
        for d in self.packed.descs:
            o = int(d["pts"])
            if self.packed.kind == _lib.KIND_CURVE:
                out.append(pts[o: o + int(d["nu"])])
            else:
                out.append(pts[o: o + int(d["nu"]) * int(d["nv"])].view(int(d["nu"]), int(d["nv"]), 3))
        return out


class NurbsSurface(_Layer):
    """A batch of NURBS surfaces with learnable control points and weights."""

    def __init__(self, surfaces, learn_knots=False, device="cuda", **plan_kw):
        super().__init__(batch.pack_surfaces(surfaces), learn_knots, True, device, **plan_kw)


class NurbsCurve(_Layer):
    """A batch of NURBS curves with learnable control points and weights."""

    def __init__(self, curves, learn_knots=False, device="cuda", **plan_kw):
        super().__init__(batch.pack_curves(curves), learn_knots, True, device, **plan_kw)


class BSplineSurface(_Layer):
    """Non-rational surfaces: every weight is 1 and only control points (and
    optionally knots) are learned."""

    def __init__(self, surfaces, learn_knots=False, device="cuda", **plan_kw):
        super().__init__(batch.pack_surfaces(surfaces), learn_knots, False, device, **plan_kw)


class BSplineCurve(_Layer):
    def __init__(self, curves, learn_knots=False, device="cuda", **plan_kw):
        super().__init__(batch.pack_curves(curves), learn_knots, False, device, **plan_kw)


def interior_knot_mask(packed: batch.Packed, device="cuda") -> torch.Tensor:
    """1 for knots that carry a gradient (interior), 0 for the p+1 end knots."""
    m = np.zeros(len(packed.knots), np.float32)
    for d in packed.descs:
        n1, p = int(d["n1"]), int(d["p"])
        m[int(d["knot_u"]) + p + 1: int(d["knot_u"]) + n1] = 1
        if packed.kind == _lib.KIND_SURFACE:
            m1, q = int(d["m1"]), int(d["q"])
            m[int(d["knot_v"]) + q + 1: int(d["knot_v"]) + m1] = 1
    return torch.from_numpy(m).to(device)
