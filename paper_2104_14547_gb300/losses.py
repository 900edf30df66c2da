"""Point-set losses of Sec. 4 on the GPU: Chamfer and Hausdorff distances
between batched point sets (nurbs_chamfer), e.g. evaluated surface points
against target point clouds."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def chamfer(P: torch.Tensor, p_sizes, Q: torch.Tensor, q_sizes, grad: bool = True, stream=None,
            bucketed: bool = True):
    """P [sum(p_sizes), 3] and Q [sum(q_sizes), 3] float32 CUDA tensors, split into
    pairs by the sizes.  Returns a dict with per-pair "cd", "hd", per-point
    "grad_cd", "grad_hd" (when grad), and the nearest-point maps "nn_p", "nn_q"
    with distances "dist_p", "dist_q".  bucketed=False takes the O(n m) gradient
    path (the same results, no scratch)."""
    dev = P.device
    p_sizes = np.asarray(p_sizes, np.int64).reshape(-1)
    q_sizes = np.asarray(q_sizes, np.int64).reshape(-1)
    if len(p_sizes) != len(q_sizes):
        raise ValueError("p_sizes and q_sizes must pair up")
    if (p_sizes < 0).any() or (q_sizes < 0).any():
        raise ValueError("set sizes must be non-negative")
    for name, X, n in (("P", P, int(p_sizes.sum())), ("Q", Q, int(q_sizes.sum()))):
        if X.numel() < 3 * n:                  # the kernels index every point of every pair
            raise ValueError(f"{name} holds {X.numel()} floats; the sizes need {3 * n}")
        if n > 0 and not X.is_cuda:
            raise ValueError(f"{name} must be on the GPU")
    count = len(p_sizes)
    p_off = torch.from_numpy(np.concatenate([[0], np.cumsum(p_sizes)]).astype(np.int64)).to(dev)
    q_off = torch.from_numpy(np.concatenate([[0], np.cumsum(q_sizes)]).astype(np.int64)).to(dev)
    P = P.contiguous().float()
    Q = Q.contiguous().float()
    np_, nq_ = int(p_sizes.sum()), int(q_sizes.sum())
    out = {"nn_p": torch.empty(max(np_, 1), dtype=torch.int32, device=dev),
           "dist_p": torch.empty(max(np_, 1), device=dev),
           "nn_q": torch.empty(max(nq_, 1), dtype=torch.int32, device=dev),
           "dist_q": torch.empty(max(nq_, 1), device=dev),
           "cd": torch.empty(max(count, 1), device=dev), "hd": torch.empty(max(count, 1), device=dev)}
    if grad:
        out["grad_cd"] = torch.empty((max(np_, 1), 3), device=dev)
        out["grad_hd"] = torch.empty((max(np_, 1), 3), device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    scratch = torch.empty(2 * np_ + nq_ + 1, dtype=torch.int32, device=dev) if (grad and bucketed) else None
    lib = _lib.load()
    _lib.check(lib.nurbs_chamfer(count, _ptr(p_off), _ptr(q_off), int(p_sizes.max(initial=0)),
                                 int(q_sizes.max(initial=0)), _ptr(P), _ptr(Q), _ptr(out["nn_p"]),
                                 _ptr(out["dist_p"]), _ptr(out["nn_q"]), _ptr(out["dist_q"]), _ptr(out["cd"]),
                                 _ptr(out["hd"]), _ptr(out.get("grad_cd")), _ptr(out.get("grad_hd")),
                                 _ptr(scratch), np_, nq_, ctypes.c_void_p(s.cuda_stream)), "nurbs_chamfer")
    out["_keep"] = (p_off, q_off, scratch)   # these stay alive until the stream has used them
    return out
