"""GPU Chamfer and Hausdorff distances (nurbs_chamfer) against the oracle.

- Nearest-point indices match exactly: both sides decide the argmin on the same
  float32 squared distances.
- Distances, losses and gradients are compared within float32 tolerances.
- Cases: ragged pairs, empty sides, ties, identical sets.
- The last test runs on surface points from the GPU forward."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2104_14547_gb300 import batch, losses, synth

pytestmark = pytest.mark.gpu


def _pairs(seed):
    rng = np.random.default_rng(seed)
    sizes = [(100, 80), (1, 5), (0, 7), (9, 0), (2000, 1500), (333, 1029), (64, 64), (50, 40)]
    Ps, Qs = [], []
    for k, (n, m) in enumerate(sizes):
        P = rng.normal(size=(n, 3)).astype(np.float32)
        Q = rng.normal(size=(m, 3)).astype(np.float32)
        if k == 6:
            Q = P.copy()                                   # identical sets: all distances 0
        if k == 7:
            Q[10:20] = Q[0:10]                             # duplicated points: ties go to the first
            P[:5] = Q[:5]
        Ps.append(P)
        Qs.append(Q)
    return Ps, Qs


def _run(Ps, Qs, bucketed=True):
    P = torch.from_numpy(np.concatenate([p.reshape(-1, 3) for p in Ps])).cuda()
    Q = torch.from_numpy(np.concatenate([q.reshape(-1, 3) for q in Qs])).cuda()
    out = losses.chamfer(P, [len(p) for p in Ps], Q, [len(q) for q in Qs], bucketed=bucketed)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items() if k != "_keep"}


def test_chamfer_matches_oracle():
    Ps, Qs = _pairs(40)
    got = _run(Ps, Qs)
    pa = qa = 0
    for k, (P, Q) in enumerate(zip(Ps, Qs)):
        cd, hd, gcd, ghd, nn_p, nn_q = O.chamfer(P, Q)
        n, m = len(P), len(Q)
        np.testing.assert_array_equal(got["nn_p"][pa: pa + n], nn_p)
        np.testing.assert_array_equal(got["nn_q"][qa: qa + m], nn_q)
        _, dp = O.nearest(P, Q)
        assert np.abs(got["dist_p"][pa: pa + n] - dp).max(initial=0) <= 1e-6 * max(1.0, dp.max(initial=0))
        assert abs(got["cd"][k] - cd) <= 1e-5 * max(1.0, cd), (k, got["cd"][k], cd)
        assert abs(got["hd"][k] - hd) <= 1e-5 * max(1.0, hd), (k, got["hd"][k], hd)
        if n:
            assert np.abs(got["grad_cd"][pa: pa + n] - gcd).max() <= 1e-4 * max(1.0, np.abs(gcd).max())
            assert np.abs(got["grad_hd"][pa: pa + n] - ghd).max() <= 1e-5
        pa += n
        qa += m


def test_chamfer_is_deterministic_and_paths_agree():
    Ps, Qs = _pairs(41)
    a, b = _run(Ps, Qs), _run(Ps, Qs)
    c = _run(Ps, Qs, bucketed=False)
    for key in ("cd", "hd", "grad_cd", "grad_hd", "nn_p", "nn_q"):
        np.testing.assert_array_equal(a[key], b[key])
        np.testing.assert_array_equal(a[key], c[key])   # bucketed and scanning gradients: same bits


def test_chamfer_of_evaluated_surfaces():
    surfs, targets = synth.bicubic_batch(42, batch=3, net=12, grid=40)
    pk, tk = batch.pack_surfaces(surfs), batch.pack_surfaces(targets)
    kn, ct, pr = batch.to_device(pk)
    _, tct, _ = batch.to_device(tk)
    S = torch.empty((pk.npts, 3), device="cuda")
    T = torch.empty((pk.npts, 3), device="cuda")
    batch.Plan.for_packed(pk).eval(kn, ct, pr, S)
    batch.Plan.for_packed(tk).eval(kn, tct, pr, T)
    sizes = [40 * 40] * 3
    out = losses.chamfer(S, sizes, T, sizes, grad=False)     # each surface against its own target
    cd = out["cd"].cpu().numpy()
    Sn, Tn = S.cpu().numpy(), T.cpu().numpy()
    for k in range(3):
        a, b = k * 1600, (k + 1) * 1600
        want = O.chamfer(Sn[a:b], Tn[a:b])[0]
        assert abs(cd[k] - want) <= 1e-5 * want
