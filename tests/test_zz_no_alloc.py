"""The allocation-free entry point nurbs_mse_fwd_bwd_noalloc, for callers that
cannot allocate device memory (its scratch is a fixed array inside the library).
It must give the results of nurbs_mse_fwd_bwd, call after call, through the
C-ABI: the same kernels, tiles and summation order, so the same bits (which is
also within the parity tolerances).  Its device-side checks must be visible
through nurbs_noalloc_get_error.  This file is collected last so that a run
stopping at the first failure has already run every other test."""
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


def _noalloc_error(lib):
    flags = ctypes.c_uint32(0)
    st = lib.nurbs_noalloc_get_error(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(flags))
    return int(st), int(flags.value)


def test_noalloc_matches_workspace_entry_point_twice():
    lib = _lib.load()
    _noalloc_error(lib)   # whatever earlier allocation-free calls left in the error word
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
        assert _noalloc_error(lib) == (0, 0)
        for key in ref:   # same kernels, tiles and summation order as the workspace call: same bits
            assert torch.equal(out[key], ref[key]), key
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


def test_noalloc_reports_device_checks():
    # samples out of order in one item: the kernels flag NURBS_ERR_ORDER in the fixed
    # array's error word, which nurbs_noalloc_get_error reads and clears
    lib = _lib.load()
    _noalloc_error(lib)
    rng = np.random.default_rng(25)
    good = synth.surface(rng, 3, 3, 10, 10, 24, 24)
    s = synth.surface(rng, 3, 3, 8, 8, 20, 20)
    unsorted = synth.Surface(s.p, s.q, s.U, s.V, s.ctrl, s.u[::-1].copy(), s.v)
    pk = batch.pack_surfaces([good, unsorted])
    plan = batch.Plan.for_packed(pk)
    kn, ct, pr = batch.to_device(pk)
    T = torch.zeros((pk.npts, 3), device="cuda")
    pts, gc, gk = torch.zeros_like(T), torch.zeros_like(ct), torch.zeros_like(kn)
    loss = torch.zeros(pk.count, device="cuda")
    for _ in range(2):   # the word collects the checks of every call until it is read
        st = _call_noalloc(lib, plan, kn, ct, pr, T, pts, gc, gk, loss, 1.0)
        assert st == 0, _lib.status_string(st)
    st, flags = _noalloc_error(lib)
    assert st == 5 and flags & (1 << 5), (st, flags)      # NURBS_ERR_ORDER
    assert _noalloc_error(lib) == (0, 0)                  # read and cleared
    assert plan.get_error() == (0, 0)                     # the plan's own workspace saw nothing
    # a clean call afterwards reports nothing
    clean = batch.pack_surfaces([good])
    cplan = batch.Plan.for_packed(clean)
    ckn, cct, cpr = batch.to_device(clean)
    CT = torch.zeros((clean.npts, 3), device="cuda")
    st = _call_noalloc(lib, cplan, ckn, cct, cpr, CT, torch.zeros_like(CT), torch.zeros_like(cct), None, None, 1.0)
    assert st == 0
    assert _noalloc_error(lib) == (0, 0)
