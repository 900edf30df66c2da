"""Tile-shape autotuner for libnurbs plans.

For a packed batch it builds one plan per candidate (warps per CTA, sample rows
per tile), times the requested entry point on the device with CUDA events (L2
flushed between repetitions) and keeps the fastest.  Results are cached per
batch signature for the life of the process.
"""
from __future__ import annotations

import hashlib

import numpy as np
import torch

from . import _lib, batch

DEFAULT_CANDIDATES = [(8, 32), (8, 64), (8, 128), (8, 256), (4, 32), (4, 64), (4, 128), (4, 256), (2, 32)]
_cache: dict = {}


def signature(packed: batch.Packed, op: str) -> str:
    h = hashlib.sha1(packed.descs.tobytes())
    h.update(op.encode())
    return h.hexdigest()


def _time(fn, reps, flush):
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def autotune(packed: batch.Packed, tensors: dict, op: str = "mse", candidates=None, reps: int = 5,
             device="cuda", max_ctas=None, budget_key=None):
    """Return (best (warps, rows), {cfg: ms}) for `op` in {"eval", "mse", "backward"}.

    tensors holds the device arrays the op needs: knots, ctrl, params and, for
    the gradient ops, target/grad_pts plus output buffers.  max_ctas, when
    given, maps a candidate's plan (uncapped) to the CTA cap it is timed under
    (the share of the GPU the plan will get when it runs beside others);
    budget_key names that budget in the result cache.
    """
    key = signature(packed, op) + repr(budget_key if max_ctas is not None else None)
    if key in _cache:
        return _cache[key]
    cands = candidates or DEFAULT_CANDIDATES
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=device)
    table = {}
    for warps, rows in cands:
        plan = batch.Plan.for_packed(packed, device=device, warps=warps, rows=rows)
        if max_ctas is not None:
            try:
                cap = int(max_ctas(plan))
            except _lib.NurbsError as e:
                if e.status != _lib.ERR_SIZE:
                    raise
                continue
            plan = batch.Plan.for_packed(packed, device=device, warps=warps, rows=rows, max_ctas=cap)
        kn, ct, pr = tensors["knots"], tensors["ctrl"], tensors["params"]
        if op == "eval":
            fn = lambda: plan.eval(kn, ct, pr, tensors["pts"])
        elif op == "backward":
            fn = lambda: plan.backward(kn, ct, pr, tensors["grad_pts"], tensors.get("grad_ctrl"),
                                       tensors.get("grad_knots"))
        else:
            fn = lambda: plan.mse_fwd_bwd(kn, ct, pr, tensors["target"], tensors.get("pts"),
                                          tensors.get("grad_ctrl"), tensors.get("grad_knots"),
                                          tensors.get("loss"))
        try:
            fn()
        except _lib.NurbsError as e:
            if e.status != _lib.ERR_SIZE:      # a shape the kernels cannot hold is skipped
                raise
            del plan
            continue
        torch.cuda.synchronize()
        table[(warps, rows)] = _time(fn, reps, flush)
        del plan
    if not table:
        raise RuntimeError("no candidate tile shape fits this batch")
    best = min(table, key=table.get)
    _cache[key] = (best, table)
    return best, table
