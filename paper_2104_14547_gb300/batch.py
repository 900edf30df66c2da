"""Host side of the hot path: pack a ragged batch into the C-ABI layout, own a
plan and its workspace, and call the libnurbs entry points on torch tensors.

This module only marshals arguments: every step of evaluation and
differentiation runs in libnurbs kernels.  PyTorch provides device memory and
the current CUDA stream.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib


@dataclass
class Packed:
    """A batch in the layout of include/nurbs.h (host numpy arrays)."""
    kind: int
    descs: np.ndarray          # structured array matching nurbs_desc
    knots: np.ndarray          # float32
    ctrl: np.ndarray           # float32 [nctrl, 4]
    params: np.ndarray         # float32
    npts: int                  # total output points

    @property
    def count(self) -> int:
        return len(self.descs)


DESC_DTYPE = np.dtype([("p", "<i4"), ("q", "<i4"), ("n1", "<i4"), ("m1", "<i4"), ("nu", "<i4"), ("nv", "<i4"),
                       ("adam_step", "<i4"), ("grad_scale", "<f4"), ("knot_u", "<i8"), ("knot_v", "<i8"), ("ctrl", "<i8"),
                       ("param_u", "<i8"), ("param_v", "<i8"), ("pts", "<i8")])
assert DESC_DTYPE.itemsize == ctypes.sizeof(_lib.Desc)


def pack_surfaces(surfs) -> Packed:
    """Pack synth.Surface-like objects (p, q, U, V, ctrl[n1, m1, 4], u, v)."""
    d = np.zeros(len(surfs), DESC_DTYPE)
    knots, ctrl, params = [], [], []
    ko = co = po = pts = 0
    for k, s in enumerate(surfs):
        n1, m1 = s.ctrl.shape[0], s.ctrl.shape[1]
        d[k] = (s.p, s.q, n1, m1, len(s.u), len(s.v), 0, 0, ko, ko + len(s.U), co, po, po + len(s.u), pts)
        knots += [np.asarray(s.U, np.float32), np.asarray(s.V, np.float32)]
        ko += len(s.U) + len(s.V)
        ctrl.append(np.asarray(s.ctrl, np.float32).reshape(-1, 4))
        co += n1 * m1
        params += [np.asarray(s.u, np.float32), np.asarray(s.v, np.float32)]
        po += len(s.u) + len(s.v)
        pts += len(s.u) * len(s.v)
    return Packed(_lib.KIND_SURFACE, d, _cat(knots), _cat(ctrl, (0, 4)), _cat(params), pts)


def pack_curves(curves) -> Packed:
    """Pack synth.Curve-like objects (p, U, ctrl[n1, 4], u)."""
    d = np.zeros(len(curves), DESC_DTYPE)
    knots, ctrl, params = [], [], []
    ko = co = po = pts = 0
    for k, c in enumerate(curves):
        n1 = c.ctrl.shape[0]
        d[k] = (c.p, 0, n1, 1, len(c.u), 1, 0, 0, ko, 0, co, po, 0, pts)
        knots.append(np.asarray(c.U, np.float32))
        ko += len(c.U)
        ctrl.append(np.asarray(c.ctrl, np.float32).reshape(-1, 4))
        co += n1
        params.append(np.asarray(c.u, np.float32))
        po += len(c.u)
        pts += len(c.u)
    return Packed(_lib.KIND_CURVE, d, _cat(knots), _cat(ctrl, (0, 4)), _cat(params), pts)


def _cat(arrs, empty_shape=(0,)):
    return np.concatenate(arrs).astype(np.float32) if arrs else np.zeros(empty_shape, np.float32)


def unpack_points(packed: Packed, pts: np.ndarray):
    """Split a flat [npts, 3] array into per-item arrays ([nu, nv, 3] or [nu, 3])."""
    pts = np.asarray(pts).reshape(-1, 3)
    out = []
    for d in packed.descs:
        o = int(d["pts"])
        if packed.kind == _lib.KIND_CURVE:
            out.append(pts[o: o + d["nu"]])
        else:
            out.append(pts[o: o + d["nu"] * d["nv"]].reshape(d["nu"], d["nv"], 3))
    return out


def unpack_ctrl(packed: Packed, arr: np.ndarray):
    arr = np.asarray(arr).reshape(-1, 4)
    out = []
    for d in packed.descs:
        o, n = int(d["ctrl"]), int(d["n1"]) * int(d["m1"])
        out.append(arr[o: o + n].reshape(d["n1"], 4) if packed.kind == _lib.KIND_CURVE
                   else arr[o: o + n].reshape(d["n1"], d["m1"], 4))
    return out


def unpack_knots(packed: Packed, arr: np.ndarray):
    """Per item: (dU, dV) for surfaces, dU for curves."""
    arr = np.asarray(arr)
    out = []
    for d in packed.descs:
        nU = int(d["n1"] + d["p"] + 1)
        dU = arr[int(d["knot_u"]): int(d["knot_u"]) + nU]
        if packed.kind == _lib.KIND_CURVE:
            out.append(dU)
        else:
            nV = int(d["m1"] + d["q"] + 1)
            out.append((dU, arr[int(d["knot_v"]): int(d["knot_v"]) + nV]))
    return out


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def item_mean_scales(descs: np.ndarray) -> np.ndarray:
    """A copy of `descs` whose items each carry grad_scale = 2 / (3 * its own point
    count): the MSE of every item is then the mean over its own points (Sec. 4,
    Eq. 12), and its gradient and Adam trajectory do not depend on which other
    items share the batch.  Items without points keep 0."""
    d = np.array(descs, dtype=DESC_DTYPE, copy=True)
    npts = d["nu"].astype(np.int64) * np.where(d["nv"] > 0, d["nv"], 1)
    d["grad_scale"] = np.where(npts > 0, (2.0 / (3.0 * np.maximum(npts, 1))).astype(np.float32), np.float32(0))
    return d


class Plan:
    """A libnurbs plan for one batch layout plus its device workspace.

    item_mean=True gives every item its own loss normalisation (item_mean_scales):
    the grad_scale argument of mse_fwd_bwd / fit_step then only applies to items
    whose descriptor scale is 0 (none, after item_mean_scales)."""

    def __init__(self, kind: int, descs: np.ndarray, device="cuda", rows: int = 0, warps: int = 0,
                 ctas_per_sm: int = 0, max_ctas: int = 0, item_mean: bool = False, workspace=None):
        self.lib = _lib.load()
        self.kind = kind
        self.descs = np.ascontiguousarray(descs, dtype=DESC_DTYPE)
        if item_mean:
            self.descs = item_mean_scales(self.descs)
        self.count = len(self.descs)
        self.warps = warps if warps > 0 else 8     # the library's default
        cfg = _lib.TileCfg(rows, warps, ctas_per_sm, max_ctas)
        h = ctypes.c_void_p()
        dptr = self.descs.ctypes.data_as(ctypes.POINTER(_lib.Desc))
        _lib.check(self.lib.nurbs_plan_create(kind, dptr, self.count, ctypes.byref(cfg), ctypes.byref(h)),
                   "nurbs_plan_create")
        self.handle = h
        self._extent = _extents(kind, self.descs)
        self.ws_bytes = int(self.lib.nurbs_plan_workspace_size(h))
        self.points = int(self.lib.nurbs_plan_points(h))
        self.tiles = int(self.lib.nurbs_plan_tiles(h))
        self.device = torch.device(device)
        if workspace is not None:
            # a caller-owned (e.g. pooled) buffer: it must be a large enough uint8 device tensor;
            # bind uploads the tables and clears the counters, the rest needs no clearing
            if (not isinstance(workspace, torch.Tensor) or workspace.dtype != torch.uint8 or not workspace.is_cuda
                    or workspace.numel() < self.ws_bytes):
                raise ValueError(f"workspace must be a uint8 device tensor of at least {self.ws_bytes} bytes")
            self.workspace = workspace
        else:
            self.workspace = torch.zeros(max(self.ws_bytes, 256), dtype=torch.uint8, device=self.device)
        _lib.check(self.lib.nurbs_plan_bind(h, _ptr(self.workspace), self.workspace.numel(), _stream()),
                   "nurbs_plan_bind")

    @classmethod
    def for_packed(cls, packed: Packed, **kw) -> "Plan":
        return cls(packed.kind, packed.descs, **kw)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                self.lib.nurbs_plan_destroy(h)
            except Exception:  # pragma: no cover - interpreter shutdown
                pass
            self.handle = None

    @property
    def ctas(self) -> int:
        return int(self.lib.nurbs_plan_ctas(self.handle))

    # ---------------------------------------------------------------- calls
    def _check(self, inputs=(), points=(), ctrl_like=(), knots_like=(), items=()):
        check_tensors(self._extent, self.count, inputs, points, ctrl_like, knots_like, items)

    def _inputs(self, knots, ctrl, params):
        return [("knots", knots, "knots"), ("ctrl", ctrl, "ctrl"), ("params", params, "params")]

    def eval(self, knots, ctrl, params, pts, stream=None):
        self._check(self._inputs(knots, ctrl, params), points=[("pts", pts)])
        if pts is None:
            raise ValueError("pts is required")
        fn = self.lib.nurbs_eval_curve if self.kind == _lib.KIND_CURVE else self.lib.nurbs_eval_surface
        _lib.check(fn(self.handle, _ptr(knots), _ptr(ctrl), _ptr(params), _ptr(pts), _stream(stream)), fn.__name__)
        return pts

    def set_knot_sigma(self, sigma: float):
        """Knot derivative of later gradient calls: 0 = almost-everywhere form,
        > 0 = the Gaussian-smoothed indicator of bandwidth sigma."""
        _lib.check(self.lib.nurbs_plan_set_knot_sigma(self.handle, ctypes.c_float(sigma)), "nurbs_plan_set_knot_sigma")

    def occupancy(self, op: str = "mse_knots"):
        """(resident CTAs per SM, dynamic shared bytes per CTA) of this plan's
        kernels for op in {"eval", "backward", "backward_knots", "mse", "mse_knots",
        "derivs"} ("mse_knots" also covers the fit step)."""
        code = {"eval": 0, "backward": 1, "backward_knots": 2, "mse": 3, "mse_knots": 4, "derivs": 5}[op]
        occ, smem = ctypes.c_int32(0), ctypes.c_int32(0)
        _lib.check(self.lib.nurbs_plan_occupancy(self.handle, code, ctypes.byref(occ), ctypes.byref(smem)),
                   "nurbs_plan_occupancy")
        return int(occ.value), int(smem.value)

    def set_grad_homogeneous(self, on: bool):
        """Control-point gradients of later calls: False = (dL/dP, dL/dw) (default),
        True = dL/dPw for Pw = (w x, w y, w z, w).  Adam in fit_step acts on (P, w) either way."""
        _lib.check(self.lib.nurbs_plan_set_grad_homogeneous(self.handle, int(bool(on))),
                   "nurbs_plan_set_grad_homogeneous")

    def eval_derivs(self, knots, ctrl, params, pts=None, du=None, dv=None, normals=None, stream=None):
        """Points with tangents and unit normals (surfaces: du, dv, normals; curves:
        the tangent goes to ``du``).  Outputs that are None are not written."""
        self._check(self._inputs(knots, ctrl, params),
                    points=[("pts", pts), ("du", du), ("dv", dv), ("normals", normals)])
        if self.kind == _lib.KIND_CURVE:
            _lib.check(self.lib.nurbs_eval_curve_derivs(self.handle, _ptr(knots), _ptr(ctrl), _ptr(params),
                                                        _ptr(pts), _ptr(du), _stream(stream)),
                       "nurbs_eval_curve_derivs")
        else:
            _lib.check(self.lib.nurbs_eval_surface_derivs(self.handle, _ptr(knots), _ptr(ctrl), _ptr(params),
                                                          _ptr(pts), _ptr(du), _ptr(dv), _ptr(normals),
                                                          _stream(stream)), "nurbs_eval_surface_derivs")
        return pts, du, dv, normals

    def backward(self, knots, ctrl, params, grad_pts, grad_ctrl=None, grad_knots=None, stream=None):
        self._check(self._inputs(knots, ctrl, params) + [("grad_pts", grad_pts, "pts3")],
                    ctrl_like=[("grad_ctrl", grad_ctrl)], knots_like=[("grad_knots", grad_knots)])
        _lib.check(self.lib.nurbs_backward(self.handle, _ptr(knots), _ptr(ctrl), _ptr(params), _ptr(grad_pts),
                                           _ptr(grad_ctrl), _ptr(grad_knots), _stream(stream)), "nurbs_backward")

    def mse_fwd_bwd(self, knots, ctrl, params, target, pts=None, grad_ctrl=None, grad_knots=None,
                    loss_items=None, grad_scale=None, stream=None):
        if grad_scale is None:
            grad_scale = 2.0 / (3.0 * max(self.points, 1))
        self._check(self._inputs(knots, ctrl, params) + [("target", target, "pts3")], points=[("pts", pts)],
                    ctrl_like=[("grad_ctrl", grad_ctrl)], knots_like=[("grad_knots", grad_knots)],
                    items=[("loss_items", loss_items)])
        _lib.check(self.lib.nurbs_mse_fwd_bwd(self.handle, _ptr(knots), _ptr(ctrl), _ptr(params), _ptr(target),
                                              _ptr(pts), _ptr(grad_ctrl), _ptr(grad_knots), _ptr(loss_items),
                                              ctypes.c_float(grad_scale), _stream(stream)), "nurbs_mse_fwd_bwd")

    def fit_step(self, knots, ctrl, params, target, adam_m, adam_v, step, lr=1e-3, betas=(0.9, 0.999),
                 eps=1e-8, pts=None, loss_items=None, grad_knots=None, grad_scale=None, stream=None):
        if grad_scale is None:
            grad_scale = 2.0 / (3.0 * max(self.points, 1))
        self._check(self._inputs(knots, ctrl, params) + [("target", target, "pts3"), ("adam_m", adam_m, "ctrl"),
                                                          ("adam_v", adam_v, "ctrl")],
                    points=[("pts", pts)], knots_like=[("grad_knots", grad_knots)], items=[("loss_items", loss_items)])
        hp = _lib.Adam(lr, betas[0], betas[1], eps)
        _lib.check(self.lib.nurbs_fit_step(self.handle, _ptr(knots), _ptr(ctrl), _ptr(params), _ptr(target),
                                           _ptr(pts), _ptr(adam_m), _ptr(adam_v), ctypes.byref(hp), int(step),
                                           ctypes.c_float(grad_scale), _ptr(loss_items), _ptr(grad_knots),
                                           _stream(stream)), "nurbs_fit_step")

    def get_error(self, stream=None):
        """(status, flags) of the device-side checks since the last call (synchronises)."""
        flags = ctypes.c_uint32(0)
        st = self.lib.nurbs_plan_get_error(self.handle, _stream(stream), ctypes.byref(flags))
        return int(st), int(flags.value)


def check_tensors(extent: dict, count: int, inputs=(), points=(), ctrl_like=(), knots_like=(), items=()):
    """Refuse, on the host, tensors the kernels would index past.  inputs are
    (name, tensor, kind) with kind one of the keys of `extent` (all required);
    points, ctrl_like, knots_like and items are (name, tensor-or-None) sized like
    the points (3 floats each), the control nets, the knot vectors and the items."""
    need = [(n, t, extent[k], True) for n, t, k in inputs]
    need += [(n, t, extent["pts3"], False) for n, t in points]
    need += [(n, t, extent["ctrl"], False) for n, t in ctrl_like]
    need += [(n, t, extent["knots"], False) for n, t in knots_like]
    need += [(n, t, count, False) for n, t in items]
    for name, t, n, required in need:
        if t is None:
            if required:
                raise ValueError(f"{name} is required")
            continue
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 tensor")
        if t.numel() < n:
            raise ValueError(f"{name} holds {t.numel()} floats; the plan's items need {n}")
        if n > 0 and not t.is_cuda:
            raise ValueError(f"{name} must be on the GPU")


def _extents(kind: int, d: np.ndarray) -> dict:
    """Floats each packed array must hold for the items of `d` (offsets + sizes)."""
    i64 = lambda x: x.astype(np.int64)
    top = lambda x: int(x.max(initial=0)) if len(x) else 0
    if kind == _lib.KIND_CURVE:
        knots = top(i64(d["knot_u"]) + d["n1"] + d["p"] + 1)
        params = top(i64(d["param_u"]) + d["nu"])
        ctrl = top(i64(d["ctrl"]) + d["n1"])
        pts = top(i64(d["pts"]) + d["nu"])
    else:
        knots = max(top(i64(d["knot_u"]) + d["n1"] + d["p"] + 1), top(i64(d["knot_v"]) + d["m1"] + d["q"] + 1))
        params = max(top(i64(d["param_u"]) + d["nu"]), top(i64(d["param_v"]) + d["nv"]))
        ctrl = top(i64(d["ctrl"]) + i64(d["n1"]) * d["m1"])
        pts = top(i64(d["pts"]) + i64(d["nu"]) * d["nv"])
    return {"knots": knots, "params": params, "ctrl": 4 * ctrl, "pts": pts, "pts3": 3 * pts}


def to_device(packed: Packed, device="cuda"):
    """(knots, ctrl, params) as device tensors."""
    dev = torch.device(device)
    return (torch.from_numpy(packed.knots).to(dev), torch.from_numpy(packed.ctrl).to(dev).contiguous(),
            torch.from_numpy(packed.params).to(dev))
