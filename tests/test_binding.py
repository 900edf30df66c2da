"""Host-side argument checks of the Python binding (no GPU needed): the extents a
plan's items index into equal the packed arrays, and tensors that are too small,
of the wrong type or layout, or on the host are refused before any kernel runs."""
import numpy as np
import pytest
import torch

from paper_2104_14547_gb300 import _lib, batch, synth


def test_extents_match_the_packed_arrays():
    rng = np.random.default_rng(0)
    surfs = [synth.surface(rng, 3, 2, 6, 7, nu, nv) for nu, nv in ((10, 12), (0, 5), (7, 0), (1, 1))]
    pk = batch.pack_surfaces(surfs)
    e = batch._extents(_lib.KIND_SURFACE, pk.descs)
    assert e["knots"] == len(pk.knots) and e["params"] == len(pk.params)
    assert e["ctrl"] == pk.ctrl.size and e["pts"] == pk.npts and e["pts3"] == 3 * pk.npts
    curves = [synth.curve(rng, p, n1, ns, knots="uniform") for p, n1, ns in ((3, 20, 50), (2, 9, 0), (5, 300, 7))]
    ck = batch.pack_curves(curves)
    e = batch._extents(_lib.KIND_CURVE, ck.descs)
    assert e["knots"] == len(ck.knots) and e["params"] == len(ck.params)
    assert e["ctrl"] == ck.ctrl.size and e["pts"] == ck.npts
    e0 = batch._extents(_lib.KIND_SURFACE, pk.descs[:0])
    assert all(v == 0 for v in e0.values())


def test_check_tensors_refuses_bad_arguments():
    ext = {"knots": 10, "params": 6, "ctrl": 16, "pts": 5, "pts3": 15}
    cpu = torch.zeros(100)
    with pytest.raises(ValueError, match="required"):
        batch.check_tensors(ext, 2, inputs=[("knots", None, "knots")])
    with pytest.raises(ValueError, match="float32"):
        batch.check_tensors(ext, 2, inputs=[("knots", torch.zeros(100, dtype=torch.float64), "knots")])
    with pytest.raises(ValueError, match="float32"):
        batch.check_tensors(ext, 2, points=[("pts", torch.zeros(10, 6)[:, ::2])])      # not contiguous
    with pytest.raises(ValueError, match="need 15"):
        batch.check_tensors(ext, 2, points=[("pts", torch.zeros(4, 3))])
    with pytest.raises(ValueError, match="need 16"):
        batch.check_tensors(ext, 2, ctrl_like=[("grad_ctrl", torch.zeros(3, 4))])
    with pytest.raises(ValueError, match="need 2"):
        batch.check_tensors(ext, 2, items=[("loss_items", torch.zeros(1))])
    with pytest.raises(ValueError, match="GPU"):
        batch.check_tensors(ext, 2, inputs=[("params", cpu, "params")])
    # optional outputs may be absent, and zero-sized needs accept any tensor
    batch.check_tensors(ext, 2, points=[("pts", None)], ctrl_like=[("grad_ctrl", None)])
    batch.check_tensors({k: 0 for k in ext}, 0, inputs=[("knots", cpu, "knots")], items=[("loss", cpu)])


def test_chamfer_refuses_bad_sizes_before_any_kernel():
    from paper_2104_14547_gb300 import losses
    P, Q = torch.zeros(10, 3), torch.zeros(8, 3)
    with pytest.raises(ValueError, match="pair up"):
        losses.chamfer(P, [5, 5], Q, [8])
    with pytest.raises(ValueError, match="non-negative"):
        losses.chamfer(P, [11, -1], Q, [4, 4])
    with pytest.raises(ValueError, match="need 33"):
        losses.chamfer(P, [5, 6], Q, [4, 4])
    with pytest.raises(ValueError, match="GPU"):
        losses.chamfer(P, [5, 5], Q, [4, 4])


def test_item_mean_scales():
    # every item's own MSE normalisation: 2 / (3 x its point count); empty items keep 0
    rng = np.random.default_rng(1)
    surfs = [synth.surface(rng, 3, 2, 6, 7, nu, nv) for nu, nv in ((10, 12), (0, 5), (7, 1))]
    pk = batch.pack_surfaces(surfs)
    d = batch.item_mean_scales(pk.descs)
    assert d["grad_scale"].dtype == np.float32
    assert d["grad_scale"][0] == np.float32(2.0 / (3 * 120)) and d["grad_scale"][1] == 0.0
    assert d["grad_scale"][2] == np.float32(2.0 / 21)
    assert np.all(pk.descs["grad_scale"] == 0.0)          # a copy: the packed batch is unchanged
    curves = [synth.curve(rng, 3, 20, n) for n in (50, 0)]
    cd = batch.item_mean_scales(batch.pack_curves(curves).descs)
    assert cd["grad_scale"][0] == np.float32(2.0 / 150) and cd["grad_scale"][1] == 0.0
