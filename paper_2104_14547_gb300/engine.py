"""Ragged batches of surfaces in one persistent, CUDA-graph-captured launch set.

A batch with mixed degrees, control nets and grids is packed once.  Items are
grouped by degree pair; each group gets its own libnurbs plan over the shared
packed arrays and a tile shape from the autotuner, and the groups' persistent
kernels run side by side on their own streams.  By default no group's CTAs are
capped: the hardware hands SM slots to whichever kernel has CTAs waiting, which
measured faster on the 1000-surface batch (875 us) than splitting the SMs by
work share (1221 us with a 16-warps-per-SM budget, 1801 us with the kernels'
real occupancy).  The whole step (forward + MSE + backward, or the fused fit
step) is captured into one CUDA graph and replayed.

`per_item_step` runs the same kernels with one launch per surface: the
unbatched form the batched engine is compared against.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib, batch, tune


# uniform tile shapes the engine also times as whole steps (all groups side by side):
# (warps, rows) or (warps, rows, CTAs per SM the shared-memory carve-up is sized for)
# (4-warp plans at 3 or 4 CTAs per SM measured 1.0-1.15 ms on the 1000-surface batch,
# against 0.69 ms for 8 x 128 at 2 per SM, and are not tried)
DEFAULT_STEP_TILES = [(8, 128), (8, 64), (4, 128), (8, 128, 2), (8, 64, 2)]


class RaggedEngine:
    """tile: one (warps, rows) for every group instead of the autotuner.
    With the autotuner, each group's shape is first tuned alone; the whole step is
    then timed (as one CUDA graph) with those shapes and with each uniform shape of
    step_candidates (default DEFAULT_STEP_TILES), and the fastest set is kept.
    budget: how a group's CTA cap is sized -- "warps" (its work share of a wave of
    16 warps per SM, what a 128-register tile kernel holds), "occupancy" (its
    share of the CTAs its kernel really fits per SM, nurbs_plan_occupancy) or
    "none" (no cap: the groups' persistent CTAs share the SMs first come, first
    served)."""

    def __init__(self, surfaces, targets_pts: np.ndarray, device="cuda", autotune=True, knots_grad=True,
                 candidates=None, tile=None, budget="none", step_candidates=None):
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.packed = batch.pack_surfaces(surfaces)
        pk = self.packed
        self.knots, self.ctrl, self.params = batch.to_device(pk, self.device)
        self.target = torch.from_numpy(np.ascontiguousarray(targets_pts, np.float32).reshape(-1, 3)).to(self.device)
        assert self.target.shape[0] == pk.npts
        self.pts = torch.empty((max(pk.npts, 1), 3), device=self.device)
        self.grad_ctrl = torch.empty_like(self.ctrl)
        self.grad_knots = torch.empty_like(self.knots) if knots_grad else None
        self.loss = torch.empty(pk.count, device=self.device)
        self.grad_scale = 2.0 / (3.0 * max(pk.npts, 1))
        self.points = pk.npts
        sms = torch.cuda.get_device_properties(self.device).multi_processor_count
        op = "mse_knots" if knots_grad else "mse"
        assert budget in ("warps", "occupancy", "none")
        # degree groups, launched heaviest first (points times the (p+1)(q+1) terms of
        # each point) so that the groups with the longest tiles do not start last
        keys = sorted(set(zip(pk.descs["p"].tolist(), pk.descs["q"].tolist())))
        work = {k: 0 for k in keys}
        for d in pk.descs:
            work[(int(d["p"]), int(d["q"]))] += int(d["nu"]) * int(d["nv"]) + 1
        keys.sort(key=lambda k: -work[k] * (k[0] + 1) * (k[1] + 1))
        total = sum(work.values())
        self._cap_fns = {}
        tuned = {}
        for k in keys:
            sel = np.nonzero((pk.descs["p"] == k[0]) & (pk.descs["q"] == k[1]))[0]
            sub = pk.descs[sel]
            # CTA budget: this group's share of a full wave of CTA slots, at least one
            # SM's worth; tile shapes are tuned under that budget
            share = work[k] / total

            def cap(plan, share=share):
                if budget == "none":
                    return 0
                per_sm = max(1, 16 // plan.warps) if budget == "warps" else max(1, plan.occupancy(op)[0])
                return max(per_sm, int(round(share * sms * per_sm)))

            self._cap_fns[k] = cap
            warps, rows = tile if tile is not None else (8, 128)
            if autotune and tile is None:
                sub_packed = batch.Packed(pk.kind, sub, pk.knots, pk.ctrl, pk.params, pk.npts)
                (warps, rows), _ = tune.autotune(sub_packed, self._tensors(), op="mse", candidates=candidates,
                                                 reps=3, device=self.device, max_ctas=cap,
                                                 budget_key=(budget, round(share, 6), sms))
            tuned[k] = (warps, rows)
        self.groups = self._build(keys, tuned)
        self.step_candidates = {}
        if autotune and tile is None:
            # Each group was tuned alone, but the groups run side by side: time the whole
            # step (one captured graph) for the per-group choice and for uniform tile
            # shapes, and keep the fastest.
            options = {"per_group": tuned}
            for t in step_candidates or DEFAULT_STEP_TILES:
                name = f"w{t[0]}r{t[1]}" + (f"c{t[2]}" if len(t) > 2 else "")
                options[name] = {k: tuple(t) for k in keys}
            best, best_ms = None, None
            for name, tiles in options.items():
                try:   # a shape whose tiles a kernel cannot hold is skipped
                    groups = self._build(keys, tiles) if name != "per_group" else self.groups
                    ms = self._time_graph(groups)
                except _lib.NurbsError as e:
                    if e.status != _lib.ERR_SIZE:
                        raise
                    continue
                self.step_candidates[name] = ms
                if best_ms is None or ms < best_ms:
                    best, best_ms = groups, ms
            self.groups = best
        self.graph = None

    def _build(self, keys, tiles):
        """One plan per degree group with the given {key: (warps, rows)} tile shapes."""
        pk = self.packed
        groups = []
        for k in keys:
            sel = np.nonzero((pk.descs["p"] == k[0]) & (pk.descs["q"] == k[1]))[0]
            sub = pk.descs[sel]
            warps, rows = tiles[k][:2]
            per_sm = tiles[k][2] if len(tiles[k]) > 2 else 0
            max_ctas = self._cap_fns[k](batch.Plan(pk.kind, sub, device=self.device, warps=warps, rows=rows,
                                                   ctas_per_sm=per_sm))
            plan = batch.Plan(pk.kind, sub, device=self.device, warps=warps, rows=rows, max_ctas=max_ctas,
                              ctas_per_sm=per_sm)
            # loss_items is indexed by the plan's own item order: one buffer per group
            groups.append(dict(key=k, items=sel, plan=plan, tile=tuple(tiles[k]), max_ctas=max_ctas,
                               loss=torch.zeros(len(sel), device=self.device),
                               stream=torch.cuda.Stream(self.device)))
        return groups

    def _time_graph(self, groups, reps: int = 3) -> float:
        """Median ms of the whole step for a set of group plans, captured in a graph
        and replayed with L2 flushed before each replay."""
        saved = self.groups
        self.groups = groups
        try:
            self.step()                               # first launch outside the capture
            torch.cuda.synchronize(self.device)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self.step()
            flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=self.device)
            ts = []
            for _ in range(reps + 1):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                g.replay()
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            del g, flush
            return float(np.median(ts[1:]))
        finally:
            self.groups = saved

    def _tensors(self):
        return dict(knots=self.knots, ctrl=self.ctrl, params=self.params, target=self.target, pts=self.pts,
                    grad_ctrl=self.grad_ctrl, grad_knots=self.grad_knots, loss=self.loss)

    # ------------------------------------------------------------------ step
    def step(self):
        """Forward + MSE + backward of every item: the groups' kernels on their own
        streams, forked from and joined back into the current stream."""
        main = torch.cuda.current_stream(self.device)
        for g in self.groups:
            g["stream"].wait_stream(main)
        for g in self.groups:
            with torch.cuda.stream(g["stream"]):
                g["plan"].mse_fwd_bwd(self.knots, self.ctrl, self.params, self.target, self.pts, self.grad_ctrl,
                                      self.grad_knots, g["loss"], self.grad_scale, stream=g["stream"])
        for g in self.groups:
            main.wait_stream(g["stream"])

    def capture(self):
        """Record one step into a CUDA graph (warm-up first, outside the capture)."""
        self.step()
        torch.cuda.synchronize(self.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step()
        torch.cuda.synchronize(self.device)
        return self.graph

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def item_losses(self) -> np.ndarray:
        """Each item's sum of squared differences, in the packed item order."""
        out = np.zeros(self.packed.count, np.float64)
        for g in self.groups:
            out[g["items"]] = g["loss"].cpu().numpy()
        return out

    def errors(self):
        out = []
        for g in self.groups:
            out.append(g["plan"].get_error()[0])
        return out


class PerItemEngine:
    """The same kernels, one plan and one launch per surface (the unbatched form),
    each with the tile shape of its degree group in the batched engine."""

    def __init__(self, eng: RaggedEngine):
        self.eng = eng
        pk = eng.packed
        tile = {}
        for g in eng.groups:
            for k in g["items"]:
                tile[int(k)] = g["tile"]
        self.plans = [batch.Plan(pk.kind, pk.descs[k: k + 1], device=eng.device, warps=tile[k][0], rows=tile[k][1],
                                 ctas_per_sm=tile[k][2] if len(tile[k]) > 2 else 0)
                      for k in range(pk.count)]

    def step(self):
        e = self.eng
        for k, p in enumerate(self.plans):
            p.mse_fwd_bwd(e.knots, e.ctrl, e.params, e.target, e.pts, e.grad_ctrl, e.grad_knots, e.loss[k:],
                          e.grad_scale)


class StreamedSteps:
    """Fused MSE steps fed from pinned host memory, with the copies overlapped.

    Each step copies its inputs (knots, control net, samples, target) host to
    device, runs the fused forward + MSE + backward, and copies its results
    (control-point and knot gradients, per-item loss) back.  Two device buffer
    sets alternate.  Step k's inputs go in on one stream while step k-1 computes
    on another and step k-2's results come back on a third, so a run of steps
    costs about max(copy in, compute + copy out) per step instead of their sum.
    """

    IN = ("knots", "ctrl", "params", "target")
    OUT = ("grad_ctrl", "grad_knots", "loss")

    def __init__(self, plan: batch.Plan, host_in: dict, host_out: dict, grad_scale: float, device="cuda"):
        self.plan = plan
        self.dev = torch.device(device)
        self.host_in, self.host_out = host_in, host_out
        self.grad_scale = float(grad_scale)
        self.bufs = []
        for _ in range(2):
            b = {k: torch.empty_like(host_in[k], device=self.dev) for k in self.IN}
            b.update({k: torch.empty_like(host_out[k], device=self.dev) for k in self.OUT})
            self.bufs.append(b)
        self.pts = torch.empty((max(plan.points, 1), 3), device=self.dev)
        self.s_in = torch.cuda.Stream(self.dev)
        self.s_cmp = torch.cuda.Stream(self.dev)
        self.s_out = torch.cuda.Stream(self.dev)
        self.ev_in = [torch.cuda.Event() for _ in range(2)]
        self.ev_cmp = [torch.cuda.Event() for _ in range(2)]
        self.ev_out = [torch.cuda.Event() for _ in range(2)]
        self.k = 0

    def step(self):
        b = self.k % 2
        buf = self.bufs[b]
        if self.k >= 2:
            self.s_in.wait_event(self.ev_cmp[b])        # step k-2 no longer reads these inputs
        with torch.cuda.stream(self.s_in):
            for key in self.IN:
                buf[key].copy_(self.host_in[key], non_blocking=True)
        self.ev_in[b].record(self.s_in)
        self.s_cmp.wait_event(self.ev_in[b])
        if self.k >= 2:
            self.s_cmp.wait_event(self.ev_out[b])       # step k-2's results have left these buffers
        self.plan.mse_fwd_bwd(buf["knots"], buf["ctrl"], buf["params"], buf["target"], self.pts,
                              buf["grad_ctrl"], buf["grad_knots"], buf["loss"], self.grad_scale, stream=self.s_cmp)
        self.ev_cmp[b].record(self.s_cmp)
        self.s_out.wait_event(self.ev_cmp[b])
        with torch.cuda.stream(self.s_out):
            for key in self.OUT:
                self.host_out[key].copy_(buf[key], non_blocking=True)
        self.ev_out[b].record(self.s_out)
        self.k += 1

    def run(self, steps: int):
        """Issue `steps` steps; returns the (start, end) events around them
        (start on the input stream, end after the last result copy)."""
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        self.s_in.wait_stream(torch.cuda.current_stream(self.dev))
        start.record(self.s_in)
        for _ in range(steps):
            self.step()
        self.s_out.wait_stream(self.s_cmp)
        end.record(self.s_out)
        return start, end
