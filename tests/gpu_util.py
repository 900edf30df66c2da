"""Helpers of the GPU parity tests: run a packed batch through libnurbs and the
same inputs through the FP64 oracle, and compare with the stated tolerances.

Tolerances (FP32 GPU path against the FP64 oracle):
  points     max |dS| <= 2e-6 x the diagonal of the control net's bounding box
  gradients  max |dg| / max |g_ref| <= 1e-3 per tensor per item
"""
import numpy as np
import torch

from oracle import oracle as O
from paper_2104_14547_gb300 import _lib, batch

S_TOL = 2e-6
G_TOL = 1e-3


def bbox_diag(ctrl):
    xyz = np.asarray(ctrl, np.float64).reshape(-1, 4)[:, :3]
    return float(np.linalg.norm(xyz.max(0) - xyz.min(0)))


def rel_inf(a, ref):
    a, ref = np.asarray(a, np.float64), np.asarray(ref, np.float64)
    den = np.abs(ref).max()
    if den == 0.0:
        return float(np.abs(a).max())
    return float(np.abs(a - ref).max() / den)


def oracle_eval(item, kind):
    if kind == _lib.KIND_CURVE:
        return O.curve_eval(item.p, item.U, item.ctrl, item.u)
    return O.surface_eval(item.p, item.q, item.U, item.V, item.ctrl, item.u, item.v)


def oracle_vjp(item, kind, g):
    if kind == _lib.KIND_CURVE:
        dc, dU = O.curve_vjp(item.p, item.U, item.ctrl, item.u, g)
        return dc, dU, None
    return O.surface_vjp(item.p, item.q, item.U, item.V, item.ctrl, item.u, item.v, g)


def pack(items, kind):
    return batch.pack_curves(items) if kind == _lib.KIND_CURVE else batch.pack_surfaces(items)


def gpu_eval(items, kind, **plan_kw):
    pk = pack(items, kind)
    plan = batch.Plan.for_packed(pk, **plan_kw)
    knots, ctrl, params = batch.to_device(pk)
    pts = torch.full((max(pk.npts, 1), 3), float("nan"), device="cuda")
    plan.eval(knots, ctrl, params, pts)
    st, flags = plan.get_error()
    assert st == 0, (st, flags)
    return pk, batch.unpack_points(pk, pts.cpu().numpy())


def check_points(items, kind, got):
    worst = 0.0
    for it, S in zip(items, got):
        ref = oracle_eval(it, kind)
        if ref.size == 0:
            continue
        err = np.abs(S.astype(np.float64) - ref).max() / max(bbox_diag(it.ctrl), 1e-30)
        worst = max(worst, err)
    assert worst <= S_TOL, worst
    return worst
