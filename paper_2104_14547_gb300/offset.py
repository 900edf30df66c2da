"""Surface offsetting with the same parameterisation (the paper's Sec. 4 CAD
application, single patches).

1. Evaluate each base surface's points S and unit normals N on its sample grid.
2. Move the points along the normals by the offset distance: T = S + d N.
3. Fit a surface to T with the base surface's degrees, knots and samples, by
   fused Adam fit steps that start from the base control net.

The direct control-point offset (every control point moved by d along the mean
normal) is kept for comparison, as the paper does.  Multi-patch normal
consolidation along shared edges is not part of this module.
"""
from __future__ import annotations

import numpy as np
import torch

from . import batch, tune


# small items (a few hundred samples) want narrow CTAs: one or two warps per item
SMALL_ITEM_CANDIDATES = tune.DEFAULT_CANDIDATES + [(1, 32), (1, 64), (2, 64)]


class OffsetFit:
    """warps, rows: the fit step's tile shape; 0 and autotune=True let the tuner
    pick it (fused MSE step timed on this batch)."""

    def __init__(self, surfaces, distance, device="cuda", warps: int = 0, rows: int = 0, autotune: bool = True):
        self.device = torch.device(device)
        pk = batch.pack_surfaces(surfaces)
        self.packed = pk
        self.knots, base, self.params = batch.to_device(pk, self.device)
        self.plan = batch.Plan.for_packed(pk, device=self.device, warps=warps, rows=rows)
        n = max(pk.npts, 1)
        self.base_pts = torch.empty((n, 3), device=self.device)
        self.normals = torch.empty((n, 3), device=self.device)
        self.plan.eval_derivs(self.knots, base, self.params, pts=self.base_pts, normals=self.normals)
        # per-point offset distance (one value per item)
        d = np.broadcast_to(np.asarray(distance, np.float32), (pk.count,))
        per_pt = np.repeat(d, (pk.descs["nu"] * pk.descs["nv"]).astype(np.int64))
        self.distance = torch.from_numpy(np.ascontiguousarray(per_pt)).to(self.device)
        self.target = torch.addcmul(self.base_pts[: pk.npts], self.distance[:, None], self.normals[: pk.npts])
        self.base_ctrl = base
        self.ctrl = base.clone()                 # the fitted net, starting from the base net
        self.adam_m = torch.zeros_like(base)
        self.adam_v = torch.zeros_like(base)
        self.loss = torch.zeros(pk.count, device=self.device)
        self.steps = 0
        if autotune and warps == 0 and rows == 0:
            scratch = dict(knots=self.knots, ctrl=base, params=self.params, target=self.target, pts=None,
                           grad_ctrl=torch.empty_like(base), grad_knots=None, loss=self.loss)
            (w, r), _ = tune.autotune(pk, scratch, op="mse", candidates=SMALL_ITEM_CANDIDATES, reps=3,
                                      device=self.device)
            self.plan = batch.Plan.for_packed(pk, device=self.device, warps=w, rows=r)
            warps, rows = w, r
        self.tile = (self.plan.warps, rows)       # rows 0: the planner's choice

    def step(self, lr: float = 2e-3):
        """One fused fit step (forward, MSE to the offset points, backward, Adam)."""
        self.steps += 1
        self.plan.fit_step(self.knots, self.ctrl, self.params, self.target, self.adam_m, self.adam_v,
                           self.steps, lr=lr, loss_items=self.loss)

    def run(self, iters: int, lr: float = 2e-3):
        for _ in range(iters):
            self.step(lr)
        return self

    def _max_dev(self, ctrl) -> np.ndarray:
        pts = torch.empty_like(self.base_pts)
        self.plan.eval(self.knots, ctrl, self.params, pts)
        dev = (pts[: self.packed.npts] - self.target).abs().amax(dim=1).cpu().numpy()
        sizes = (self.packed.descs["nu"] * self.packed.descs["nv"]).astype(np.int64)
        out = np.zeros(self.packed.count)
        for k, (a, b) in enumerate(zip(np.cumsum(sizes) - sizes, np.cumsum(sizes))):
            out[k] = dev[a:b].max() if b > a else 0.0
        return out

    def deviation(self) -> np.ndarray:
        """Per item: max |S_fit - T| over its samples (largest coordinate error)."""
        return self._max_dev(self.ctrl)

    def control_point_offset_deviation(self) -> np.ndarray:
        """The same for the direct offset: each control net moved by d along the
        mean of its surface's normals."""
        pk = self.packed
        cp = self.base_ctrl.clone()
        nrm = self.normals[: pk.npts].cpu().numpy()
        ctrl_np = cp.cpu().numpy()
        sizes = (pk.descs["nu"] * pk.descs["nv"]).astype(np.int64)
        starts = np.cumsum(sizes) - sizes
        d = self.distance.cpu().numpy()
        for k, desc in enumerate(pk.descs):
            if sizes[k] == 0:
                continue
            mn = nrm[starts[k]: starts[k] + sizes[k]].mean(0)
            mn /= max(np.linalg.norm(mn), 1e-30)
            c0, nc = int(desc["ctrl"]), int(desc["n1"] * desc["m1"])
            ctrl_np[c0: c0 + nc, :3] += d[starts[k]] * mn
        return self._max_dev(torch.from_numpy(ctrl_np).to(self.device))

