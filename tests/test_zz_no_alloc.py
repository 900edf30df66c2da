"""The allocation-free entry point nurbs_mse_fwd_bwd_noalloc, for callers that
cannot allocate device memory (its scratch is a fixed array inside the library).
It must give the results of nurbs_mse_fwd_bwd, call after call, through the
C-ABI.  This file is collected last so that a run stopping at the first failure
has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from gpu_util import G_TOL, S_TOL, bbox_diag, rel_inf
from oracle import oracle as O
from paper_2104_14547_gb300 import _lib, batch, synth

pytestmark = pytest.mark.gpu

NOALLOC_LIMIT = 8 << 20   # NURBS_NOALLOC_SCRATCH_BYTES in include/nurbs.h


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _call_noalloc(lib, plan, kn, ct, pr, T, pts, gc, gk, loss, scale):
    return lib.nurbs_mse_fwd_bwd_noalloc(plan.handle, _ptr(kn), _ptr(ct), _ptr(pr), _ptr(T), _ptr(pts), _ptr(gc),
                                         _ptr(gk), _ptr(loss), ctypes.c_float(scale),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_workspace_entry_point_twice():
    lib = _lib.load()
    surfs, tg = synth.bicubic_batch(21, batch=12, net=16, grid=70)
    surfs.append(synth.surface(np.random.default_rng(22), 2, 4, 9, 11, 33, 150))   # another degree group, 2 warps
    tg.append(synth.twin_net(np.random.default_rng(23), surfs[-1]))
    T = np.concatenate([O.surface_eval(t.p, t.q, t.U, t.V, t.ctrl, t.u, t.v).reshape(-1, 3) for t in tg])
    pk = batch.pack_surfaces(surfs)
    plan = batch.Plan.for_packed(pk)
    assert plan.ws_bytes <= NOALLOC_LIMIT
    kn, ct, pr = batch.to_device(pk)
    Td = torch.from_numpy(T.astype(np.float32)).cuda()
    scale = 2.0 / (3 * pk.npts)

    ref = dict(pts=torch.zeros((pk.npts, 3), device="cuda"), gc=torch.zeros_like(ct), gk=torch.zeros_like(kn),
               loss=torch.zeros(pk.count, device="cuda"))
    plan.mse_fwd_bwd(kn, ct, pr, Td, ref["pts"], ref["gc"], ref["gk"], ref["loss"], scale)
    assert plan.get_error()[0] == 0

    for call in range(2):   # the shared scratch keeps the previous call's contents
        out = dict(pts=torch.full((pk.npts, 3), float("nan"), device="cuda"), gc=torch.full_like(ct, float("nan")),
                   gk=torch.full_like(kn, float("nan")), loss=torch.full((pk.count,), float("nan"), device="cuda"))
        st = _call_noalloc(lib, plan, kn, ct, pr, Td, out["pts"], out["gc"], out["gk"], out["loss"], scale)
        assert st == 0, _lib.status_string(st)
        torch.cuda.synchronize()
        S_ref = batch.unpack_points(pk, ref["pts"].cpu().numpy())
        S_new = batch.unpack_points(pk, out["pts"].cpu().numpy())
        for s, a, b in zip(surfs, S_ref, S_new):
            assert np.abs(a.astype(np.float64) - b).max() <= S_TOL * bbox_diag(s.ctrl)
        for a, b in zip(batch.unpack_ctrl(pk, ref["gc"].cpu().numpy()), batch.unpack_ctrl(pk, out["gc"].cpu().numpy())):
            assert rel_inf(b, a) <= G_TOL
        for (ua, va), (ub, vb) in zip(batch.unpack_knots(pk, ref["gk"].cpu().numpy()),
                                      batch.unpack_knots(pk, out["gk"].cpu().numpy())):
            assert rel_inf(ub, ua) <= G_TOL and rel_inf(vb, va) <= G_TOL
        np.testing.assert_allclose(out["loss"].cpu().numpy(), ref["loss"].cpu().numpy(), rtol=1e-5)


def test_noalloc_rejects_plans_beyond_its_scratch():
    lib = _lib.load()
    surfs, _ = synth.bicubic_batch(24, batch=64, net=32, grid=128)
    pk = batch.pack_surfaces(surfs)
    plan = batch.Plan.for_packed(pk)
    assert plan.ws_bytes > NOALLOC_LIMIT
    kn, ct, pr = batch.to_device(pk)
    buf = torch.zeros((pk.npts, 3), device="cuda")
    st = _call_noalloc(lib, plan, kn, ct, pr, buf, None, torch.zeros_like(ct), None, None, 1.0)
    assert st == 6   # NURBS_ERR_WORKSPACE, before any GPU work
