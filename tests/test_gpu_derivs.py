"""GPU tangents and normals (nurbs_eval_surface_derivs / nurbs_eval_curve_derivs)
against the FP64 oracle: surfaces of mixed degrees, tile shapes and ragged
grids, curves on both kernel paths, the exact cylinder, edge cases."""
import json
import os

import numpy as np
import pytest
import torch

from gpu_util import S_TOL, bbox_diag, pack
from oracle import oracle as O
from paper_2104_14547_gb300 import _lib, batch, synth

pytestmark = pytest.mark.gpu
SURF, CURVE = _lib.KIND_SURFACE, _lib.KIND_CURVE
D_TOL = 1e-4    # tangents: max abs error / max |tangent| of the item
N_TOL = 2e-4    # unit normals: max abs error
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _surfaces(seed):
    rng = np.random.default_rng(seed)
    specs = [(3, 3, 16, 16, 64, 64), (2, 4, 9, 11, 40, 130), (5, 1, 8, 3, 33, 7), (1, 2, 2, 5, 5, 300),
             (4, 5, 30, 12, 129, 31), (3, 2, 6, 6, 1, 1)]
    return [synth.surface(rng, p, q, n1, m1, nu, nv, knots="random", min_gap=1e-3) for p, q, n1, m1, nu, nv in specs]


def _run_surface(items, **plan_kw):
    pk = pack(items, SURF)
    plan = batch.Plan.for_packed(pk, **plan_kw)
    kn, ct, pr = batch.to_device(pk)
    n = max(pk.npts, 1)
    outs = [torch.full((n, 3), float("nan"), device="cuda") for _ in range(4)]
    plan.eval_derivs(kn, ct, pr, *outs)
    assert plan.get_error()[0] == 0
    return pk, [batch.unpack_points(pk, o.cpu().numpy()) for o in outs]


def _check_surface(items, got):
    S, Su, Sv, Nrm = got
    for k, it in enumerate(items):
        rS, rSu, rSv, rN = O.surface_derivs(it.p, it.q, it.U, it.V, it.ctrl, it.u, it.v)
        if rS.size == 0:
            continue
        assert np.abs(S[k] - rS).max() <= S_TOL * bbox_diag(it.ctrl), k
        for g, r in ((Su[k], rSu), (Sv[k], rSv)):
            assert np.abs(g - r).max() <= D_TOL * max(np.abs(r).max(), 1e-30), (k, np.abs(g - r).max())
        assert np.abs(Nrm[k] - rN).max() <= N_TOL, (k, np.abs(Nrm[k] - rN).max())


@pytest.mark.parametrize("warps,rows", [(0, 0), (4, 32), (8, 128), (2, 7)])
def test_surface_tangents_normals(warps, rows):
    items = _surfaces(20)
    _, got = _run_surface(items, warps=warps, rows=rows)
    _check_surface(items, got)


def test_surface_derivs_partial_outputs_and_points_unchanged():
    items = _surfaces(21)[:3]
    pk = pack(items, SURF)
    plan = batch.Plan.for_packed(pk)
    kn, ct, pr = batch.to_device(pk)
    pts = torch.empty((pk.npts, 3), device="cuda")
    plan.eval(kn, ct, pr, pts)
    pts2 = torch.empty_like(pts)
    nrm = torch.empty_like(pts)
    plan.eval_derivs(kn, ct, pr, pts=pts2, normals=nrm)      # no tangent buffers
    assert torch.equal(pts, pts2)                              # same points as the plain forward
    got = batch.unpack_points(pk, nrm.cpu().numpy())
    for k, it in enumerate(items):
        _, _, _, rN = O.surface_derivs(it.p, it.q, it.U, it.V, it.ctrl, it.u, it.v)
        assert np.abs(got[k] - rN).max() <= N_TOL


def test_cylinder_normals_are_radial():
    g = json.load(open(os.path.join(GOLDEN, "rational_circle.json")))
    c, cy = g["full_circle"], g["cylinder"]
    circ = np.array(c["ctrl"], dtype=np.float32)
    net = np.zeros((len(circ), 2, 4), np.float32)
    for j, z in enumerate((0.0, 1.0)):
        net[:, j, :] = circ
        net[:, j, 2] = z
    s = synth.Surface(2, 1, np.array(c["U"], np.float32), np.array(cy["V"], np.float32), net,
                      synth.uniform_params(97), synth.uniform_params(9))
    _, (S, Su, Sv, Nrm) = _run_surface([s])
    radial = S[0].copy()
    radial[..., 2] = 0
    radial /= np.linalg.norm(radial, axis=-1, keepdims=True)
    assert np.abs(np.abs(np.einsum("abk,abk->ab", Nrm[0], radial)) - 1.0).max() <= 1e-5
    assert np.abs(Sv[0] - np.array([0, 0, 1.0])).max() <= 1e-5


def test_curve_tangents_both_paths():
    rng = np.random.default_rng(22)
    specs = [(3, 64, 1024), (1, 2, 5), (2, 17, 300), (5, 6, 1), (3, 300, 700), (4, 40, 0), (2, 60, 4)]
    curves = [synth.curve(rng, p, n1, nu, min_gap=min(1e-3, 0.01 / n1)) for p, n1, nu in specs]
    pk = pack(curves, CURVE)
    plan = batch.Plan.for_packed(pk)
    kn, ct, pr = batch.to_device(pk)
    n = max(pk.npts, 1)
    pts, tan = torch.full((n, 3), float("nan"), device="cuda"), torch.full((n, 3), float("nan"), device="cuda")
    plan.eval_derivs(kn, ct, pr, pts=pts, du=tan)
    assert plan.get_error()[0] == 0
    P, T = batch.unpack_points(pk, pts.cpu().numpy()), batch.unpack_points(pk, tan.cpu().numpy())
    for k, c in enumerate(curves):
        rC, rT = O.curve_derivs(c.p, c.U, c.ctrl, c.u)
        if rC.size == 0:
            continue
        assert np.abs(P[k] - rC).max() <= S_TOL * bbox_diag(c.ctrl), k
        assert np.abs(T[k] - rT).max() <= D_TOL * np.abs(rT).max(), (k, np.abs(T[k] - rT).max())


def test_derivs_argument_errors():
    items = _surfaces(23)[:1]
    pk = pack(items, SURF)
    plan = batch.Plan.for_packed(pk)
    kn, ct, pr = batch.to_device(pk)
    with pytest.raises(_lib.NurbsError):
        plan.eval_derivs(kn, ct, pr)                 # every output missing
