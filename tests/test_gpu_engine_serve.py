"""Ragged batches through the multi-stream, CUDA-graph engine; the per-surface
form; and the continuous-batching server (results identical alone and in the mix)."""
import numpy as np
import pytest
import torch

from gpu_util import G_TOL, S_TOL, bbox_diag, rel_inf
from oracle import oracle as O
from paper_2104_14547_gb300 import batch, engine, serve, synth

pytestmark = pytest.mark.gpu


def _ragged(seed, n):
    surfs, tg = synth.ragged_batch(seed, batch=n, deg=(2, 5), net=(8, 24), grid=(20, 70))
    T = np.concatenate([O.surface_eval(t.p, t.q, t.U, t.V, t.ctrl, t.u, t.v).reshape(-1, 3) for t in tg])
    return surfs, T


def test_engine_graph_matches_oracle_and_eager():
    surfs, T = _ragged(41, 14)
    eng = engine.RaggedEngine(surfs, T, candidates=[(4, 16), (4, 32), (2, 32)])
    assert len(eng.groups) > 1
    eng.step()
    torch.cuda.synchronize()
    eager = (eng.pts.clone(), eng.grad_ctrl.clone(), eng.grad_knots.clone())
    eng.capture()
    eng.pts.zero_(); eng.grad_ctrl.zero_(); eng.grad_knots.zero_()
    eng.replay()
    torch.cuda.synchronize()
    assert all(e == 0 for e in eng.errors())
    for a, b in zip(eager, (eng.pts, eng.grad_ctrl, eng.grad_knots)):
        assert torch.equal(a, b)
    pk = eng.packed
    S = batch.unpack_points(pk, eng.pts.cpu().numpy())
    dc = batch.unpack_ctrl(pk, eng.grad_ctrl.cpu().numpy())
    dk = batch.unpack_knots(pk, eng.grad_knots.cpu().numpy())
    Tk = batch.unpack_points(pk, T)
    losses = eng.item_losses()
    for k, s in enumerate(surfs):
        ref = O.surface_eval(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v)
        assert np.abs(S[k] - ref).max() <= S_TOL * bbox_diag(s.ctrl)
        L, g = O.mse(ref, Tk[k].astype(np.float64), 3 * pk.npts)
        rc, rU, rV = O.surface_vjp(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v, g)
        assert rel_inf(dc[k], rc) <= G_TOL
        assert rel_inf(dk[k][0], rU) <= G_TOL and rel_inf(dk[k][1], rV) <= G_TOL
        assert abs(losses[k] - L * 3 * pk.npts) <= 1e-4 * max(L * 3 * pk.npts, 1e-12)


def test_per_item_form_matches_batched():
    surfs, T = _ragged(42, 6)
    eng = engine.RaggedEngine(surfs, T, autotune=False)
    eng.step()
    torch.cuda.synchronize()
    ref = eng.grad_ctrl.clone()
    per = engine.PerItemEngine(eng)
    eng.grad_ctrl.zero_()
    per.step()
    torch.cuda.synchronize()
    # same tile shape alone and in the batch: identical bits
    assert torch.equal(ref, eng.grad_ctrl)


def _wait(r):
    assert r.done.wait(timeout=60.0), "request not served within 60 s"
    assert r.error is None, r.error


def test_server_results_same_alone_and_in_the_mix():
    rng = np.random.default_rng(43)
    srv = serve.Server(hbm_fraction=0.02, max_wave=64, out_points=1 << 20)
    mids, surfs = [], []
    for k in range(10):
        p, q = int(rng.integers(2, 6)), int(rng.integers(2, 6))
        s = synth.surface(rng, p, q, int(rng.integers(p + 1, 20)), int(rng.integers(q + 1, 20)),
                          int(rng.integers(8, 60)), int(rng.integers(8, 60)))
        t = synth.twin_net(rng, s)
        mids.append(srv.register(s, O.surface_eval(t.p, t.q, t.U, t.V, t.ctrl, t.u, t.v)))
        surfs.append(s)
    assert all(m is not None for m in mids)
    srv.start()
    try:
        # alone: one request at a time
        alone = {}
        for m in mids[:4]:
            r = srv.submit(serve.Request("eval", m))
            _wait(r)
            alone[m] = r.result
        # in the mix: evaluations of those models among fit steps on the others
        reqs = [srv.submit(serve.Request("fit", m)) for m in mids[4:]]
        reqs += [srv.submit(serve.Request("eval", m)) for m in mids[:4]]
        for r in reqs:
            _wait(r)
        for r in reqs[len(mids) - 4:]:
            assert np.array_equal(r.result, alone[r.model])
            s = surfs[mids.index(r.model)]
            ref = O.surface_eval(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v)
            assert np.abs(r.result - ref).max() <= S_TOL * bbox_diag(s.ctrl)
        # fit steps lower each model's loss
        first = {r.model: r.result for r in reqs[: len(mids) - 4]}
        again = [srv.submit(serve.Request("fit", m)) for m in mids[4:] for _ in range(20)]
        for r in again:
            _wait(r)
        last = {r.model: r.result for r in again}
        assert all(last[m] < first[m] for m in mids[4:])
    finally:
        srv.stop()


def test_streamed_steps_match_direct_step():
    surfs, targets = synth.bicubic_batch(44, batch=5, net=10, grid=33)
    pk, tk = batch.pack_surfaces(surfs), batch.pack_surfaces(targets)
    kn, ct, pr = batch.to_device(pk)
    _, tct, _ = batch.to_device(tk)
    plan = batch.Plan.for_packed(pk)
    T = torch.empty((pk.npts, 3), device="cuda")
    batch.Plan.for_packed(tk).eval(kn, tct, pr, T)
    scale = 2.0 / (3.0 * pk.npts)
    gc, gk, loss = torch.empty_like(ct), torch.empty_like(kn), torch.empty(pk.count, device="cuda")
    plan.mse_fwd_bwd(kn, ct, pr, T, None, gc, gk, loss, scale)
    host_in = {"knots": kn.cpu().pin_memory(), "ctrl": ct.cpu().pin_memory(), "params": pr.cpu().pin_memory(),
               "target": T.cpu().pin_memory()}
    host_out = {"grad_ctrl": torch.empty_like(gc, device="cpu").pin_memory(),
                "grad_knots": torch.empty_like(gk, device="cpu").pin_memory(),
                "loss": torch.empty_like(loss, device="cpu").pin_memory()}
    runner = engine.StreamedSteps(plan, host_in, host_out, scale)
    _, end = runner.run(5)
    end.synchronize()
    assert torch.equal(host_out["grad_ctrl"], gc.cpu())
    assert torch.equal(host_out["grad_knots"], gk.cpu())
    assert torch.equal(host_out["loss"], loss.cpu())


def test_engine_budgets_change_no_bits():
    # CTA caps change only which SM runs a tile, never the result
    surfs, T = _ragged(43, 24)
    outs = []
    for budget in ("none", "warps", "occupancy"):
        eng = engine.RaggedEngine(surfs, T, tile=(4, 32), budget=budget)
        assert len(eng.groups) > 1
        eng.replay()
        torch.cuda.synchronize()
        assert all(e == 0 for e in eng.errors())
        if budget != "none":
            assert all(g["max_ctas"] > 0 for g in eng.groups)
        outs.append((eng.pts.clone(), eng.grad_ctrl.clone(), eng.grad_knots.clone(), eng.item_losses()))
    for o in outs[1:]:
        for a, b in zip(outs[0][:3], o[:3]):
            assert torch.equal(a, b)
        assert np.array_equal(outs[0][3], o[3])


def test_plan_occupancy_reports_what_launches():
    surfs, _ = synth.bicubic_batch(0, 4, 32, 128)
    pk = batch.pack_surfaces(surfs)
    plan = batch.Plan.for_packed(pk, warps=8, rows=128)
    occ, smem = plan.occupancy("mse_knots")
    assert occ >= 1 and 48 * 1024 < smem <= 227 * 1024
    occ_e, smem_e = plan.occupancy("eval")
    assert smem_e < smem and occ_e >= occ          # the forward has no shared adjoint
    assert plan.occupancy("derivs")[1] >= smem_e
    # a plan as wide as the GPU holds: the grid of a long batch is occupancy x SMs
    bpk = batch.pack_surfaces(synth.bicubic_batch(1, 1200, 8, 64)[0])
    big = batch.Plan.for_packed(bpk, warps=8, rows=64)
    kn, ct, pr = batch.to_device(bpk)
    pts = torch.empty((big.points, 3), device="cuda")
    big.eval(kn, ct, pr, pts)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert big.ctas == min(big.tiles, big.occupancy("eval")[0] * sms)
    curves, _ = synth.cubic_curve_batch(0, 8, 64, 256)
    cplan = batch.Plan.for_packed(batch.pack_curves(curves))
    assert cplan.occupancy("eval")[0] == 8 and cplan.occupancy("mse")[0] == 4


def _server_models(srv, seed, n, twins=0):
    """n random ragged-shaped models (and `twins` more that repeat the first ones:
    same surface, same target), registered on srv."""
    rng = np.random.default_rng(seed)
    mids, surfs, targets = [], [], []
    for k in range(n):
        p, q = int(rng.integers(2, 6)), int(rng.integers(2, 6))
        s = synth.surface(rng, p, q, int(rng.integers(p + 1, 20)), int(rng.integers(q + 1, 20)),
                          int(rng.integers(8, 60)), int(rng.integers(8, 60)))
        t = synth.twin_net(rng, s)
        surfs.append(s)
        targets.append(O.surface_eval(t.p, t.q, t.U, t.V, t.ctrl, t.u, t.v))
    for k in range(n + twins):
        mids.append(srv.register(surfs[k % n], targets[k % n]))
    assert all(m is not None for m in mids)
    return mids, surfs, targets


def _model_state(srv, mid):
    m = srv.models[mid]
    n = m.n1 * m.m1
    return (srv.ctrl[m.ctrl: m.ctrl + n].cpu().numpy(), srv.adam_m[m.ctrl: m.ctrl + n].cpu().numpy(),
            srv.adam_v[m.ctrl: m.ctrl + n].cpu().numpy())


def test_server_fits_same_alone_and_in_the_mix():
    # models 0..3 fit alone (one request at a time); their twins 8..11 fit in the mix,
    # interleaved with evaluations and fit steps of models 4..7, several per wave
    srv = serve.Server(hbm_fraction=0.02, max_wave=64, out_points=1 << 20)
    mids, surfs, targets = _server_models(srv, 45, 8, twins=4)
    alone_ids, other_ids, mix_ids = mids[:4], mids[4:8], mids[8:12]
    k_steps = 4
    srv.start()
    try:
        alone_loss = {m: [] for m in alone_ids}
        for _ in range(k_steps):
            for m in alone_ids:
                r = srv.submit(serve.Request("fit", m))
                _wait(r)
                alone_loss[m].append(r.result)
        mix_reqs = {m: [] for m in mix_ids}
        reqs = []
        for step in range(k_steps):
            for j, m in enumerate(mix_ids):
                reqs.append(srv.submit(serve.Request("eval", other_ids[j])))
                r = srv.submit(serve.Request("fit", m))
                mix_reqs[m].append(r)
                reqs.append(r)
                reqs.append(srv.submit(serve.Request("fit", other_ids[(j + step) % 4])))
        for r in reqs:
            _wait(r)
        for a, b in zip(alone_ids, mix_ids):
            assert [r.result for r in mix_reqs[b]] == alone_loss[a]
            for x, y in zip(_model_state(srv, a), _model_state(srv, b)):
                assert np.array_equal(x, y)
    finally:
        srv.stop()


def test_server_first_fit_matches_oracle_adam():
    # one fit request = Adam step 1 on the gradient of the model's own mean squared error
    srv = serve.Server(hbm_fraction=0.02, max_wave=64, out_points=1 << 20, lr=1e-3)
    mids, surfs, targets = _server_models(srv, 46, 3)
    srv.start()
    try:
        reqs = [srv.submit(serve.Request("fit", m)) for m in mids]
        for r in reqs:
            _wait(r)
        for m, s, T, r in zip(mids, surfs, targets, reqs):
            S = O.surface_eval(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v)
            Tf = np.asarray(T, np.float32).astype(np.float64)
            L, g = O.mse(S, Tf, 3 * s.npts)
            assert abs(r.result - L) <= 1e-4 * L
            dc, _, _ = O.surface_vjp(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v, g)
            th, _, _ = O.adam(s.ctrl.astype(np.float64), dc, np.zeros_like(dc), np.zeros_like(dc), 1, lr=1e-3)
            after = _model_state(srv, m)[0].reshape(th.shape)
            # step 1 moves each component by lr * sign(g): compare where the sign is sure
            sure = np.abs(dc) > 1e-2 * np.abs(dc).max()
            assert np.abs(after - th)[sure].max(initial=0.0) <= 1e-6 + 1e-6 * np.abs(th).max()
    finally:
        srv.stop()


def test_server_checkpoint_restore_continues_bit_for_bit():
    srv = serve.Server(hbm_fraction=0.02, max_wave=64, out_points=1 << 20)
    mids, _, _ = _server_models(srv, 47, 5)
    srv.start()
    try:
        for _ in range(3):
            rs = [srv.submit(serve.Request("fit", m)) for m in mids]
            for r in rs:
                _wait(r)
        ck = srv.checkpoint()
        rs = [srv.submit(serve.Request("fit", m)) for m in mids]
        for r in rs:
            _wait(r)
        first = [(r.result, _model_state(srv, r.model)) for r in rs]
        srv.restore(ck)
        assert all(srv.models[m].steps == 3 for m in mids)
        rs = [srv.submit(serve.Request("fit", m)) for m in mids]
        for r in rs:
            _wait(r)
        for (loss, st), r in zip(first, rs):
            assert r.result == loss
            for x, y in zip(st, _model_state(srv, r.model)):
                assert np.array_equal(x, y)
    finally:
        srv.stop()


def test_server_cancelled_request_never_runs():
    # a request withdrawn before admission completes as cancelled and leaves its model untouched
    srv = serve.Server(hbm_fraction=0.02, max_wave=64, out_points=1 << 20)
    mids, _, _ = _server_models(srv, 48, 2)
    before = _model_state(srv, mids[0])
    r = serve.Request("fit", mids[0])
    r.cancel()
    srv.submit(r)                       # queued before the scheduler starts
    srv.start()
    try:
        assert r.done.wait(timeout=30.0)
        assert r.error == "cancelled"
        ok = srv.submit(serve.Request("eval", mids[1]))
        _wait(ok)
        assert srv.models[mids[0]].steps == 0
        for x, y in zip(before, _model_state(srv, mids[0])):
            assert np.array_equal(x, y)
    finally:
        srv.stop()


def test_server_admission_refuses_when_arena_is_full():
    # a tiny HBM share: registration succeeds while the arena has room, then refuses
    srv = serve.Server(hbm_fraction=1e-9, max_wave=16, out_points=1 << 16)
    rng = np.random.default_rng(49)
    s = synth.surface(rng, 3, 3, 32, 32, 64, 64)
    T = np.zeros((64, 64, 3))
    got = [srv.register(s, T) for _ in range(80)]
    admitted = [m for m in got if m is not None]
    assert 0 < len(admitted) < len(got)
    assert all(m is None for m in got[len(admitted):])   # once full, every later model is refused


def test_server_eval_into_caller_buffer():
    # an evaluation with a caller-provided output array fills it with the same bits
    srv = serve.Server(hbm_fraction=0.02, max_wave=64, out_points=1 << 20)
    mids, surfs, _ = _server_models(srv, 50, 3)
    srv.start()
    try:
        for m, s in zip(mids, surfs):
            a = srv.submit(serve.Request("eval", m))
            _wait(a)
            buf = np.full(s.npts * 3, np.nan, np.float32)
            b = srv.submit(serve.Request("eval", m, out=buf))
            _wait(b)
            assert b.result is buf
            assert np.array_equal(buf.reshape(a.result.shape), a.result)
    finally:
        srv.stop()


def test_two_ctas_per_sm_carve_up_same_results():
    # single-tile degree-5 items 225 to 256 samples wide with 36..44-point nets: their
    # tables and shared adjoints need more shared memory than two 8-warp CTAs can share;
    # a plan asked for 2 CTAs per SM trims its carve-up (adjoints through the workspace,
    # then no staged net) and gives the same results
    rng = np.random.default_rng(52)
    surfs, tg = [], []
    for _ in range(10):
        n1, m1 = (int(x) for x in rng.integers(36, 45, size=2))
        s = synth.surface(rng, 5, 5, n1, m1, int(rng.integers(96, 129)), int(rng.integers(225, 257)))
        surfs.append(s)
        tg.append(synth.twin_net(rng, s))
    T = np.concatenate([O.surface_eval(t.p, t.q, t.U, t.V, t.ctrl, t.u, t.v).reshape(-1, 3) for t in tg])
    pk = batch.pack_surfaces(surfs)
    kn, ct, pr = batch.to_device(pk)
    Td = torch.from_numpy(T.astype(np.float32)).cuda()
    outs, occs = [], []
    for per_sm in (0, 2):
        plan = batch.Plan.for_packed(pk, warps=8, rows=128, ctas_per_sm=per_sm)
        occs.append(plan.occupancy("mse_knots")[0])
        pts, gc, gk = torch.empty_like(Td), torch.empty_like(ct), torch.empty_like(kn)
        loss = torch.empty(pk.count, device="cuda")
        plan.mse_fwd_bwd(kn, ct, pr, Td, pts, gc, gk, loss, 2.0 / (3 * pk.npts))
        assert plan.get_error()[0] == 0
        outs.append((pts, gc, gk, loss))
    assert occs[0] == 1 and occs[1] == 2, occs
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    # and both agree with the oracle on a sample of items
    S = batch.unpack_points(pk, outs[1][0].cpu().numpy())
    dc = batch.unpack_ctrl(pk, outs[1][1].cpu().numpy())
    Tk = batch.unpack_points(pk, T)
    for k in (0, 5, 9):
        s = surfs[k]
        ref = O.surface_eval(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v)
        assert np.abs(S[k] - ref).max() <= S_TOL * bbox_diag(s.ctrl)
        _, g = O.mse(ref, Tk[k].astype(np.float64), 3 * pk.npts)
        rc, _, _ = O.surface_vjp(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v, g)
        assert rel_inf(dc[k], rc) <= G_TOL


def test_plan_at_the_48k_shared_memory_edge_launches():
    # a serving wave's fit plan whose carve-up came to exactly 48 KB: with the kernels'
    # few bytes of static shared memory that is over the default per-block limit, so the
    # kernel's limit must be raised before launch (a wave like this once failed with
    # "item exceeds a kernel limit")
    rng = np.random.default_rng(61)
    surfs = [synth.surface(rng, 4, 3, 45, 40, 221, 200), synth.surface(rng, 4, 5, 58, 8, 110, 114)]
    tg = [synth.twin_net(rng, s) for s in surfs]
    T = np.concatenate([O.surface_eval(t.p, t.q, t.U, t.V, t.ctrl, t.u, t.v).reshape(-1, 3) for t in tg])
    pk = batch.pack_surfaces(surfs)
    kn, ct, pr = batch.to_device(pk)
    Td = torch.from_numpy(T.astype(np.float32)).cuda()
    plan = batch.Plan.for_packed(pk, warps=4, rows=32)
    for op in ("eval", "mse", "mse_knots"):
        assert plan.occupancy(op)[0] >= 1, op
    pts, gc, gk = torch.empty_like(Td), torch.empty_like(ct), torch.empty_like(kn)
    loss = torch.empty(pk.count, device="cuda")
    plan.mse_fwd_bwd(kn, ct, pr, Td, pts, gc, gk, loss, 2.0 / (3 * pk.npts))
    m, v = torch.zeros_like(ct), torch.zeros_like(ct)
    ct2 = ct.clone()
    plan.fit_step(kn, ct2, pr, Td, m, v, 1, loss_items=loss)
    torch.cuda.synchronize()
    assert plan.get_error()[0] == 0
    S = batch.unpack_points(pk, pts.cpu().numpy())
    dc = batch.unpack_ctrl(pk, gc.cpu().numpy())
    Tk = batch.unpack_points(pk, T)
    for k, s in enumerate(surfs):
        ref = O.surface_eval(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v)
        assert np.abs(S[k] - ref).max() <= S_TOL * bbox_diag(s.ctrl)
        _, g = O.mse(ref, Tk[k].astype(np.float64), 3 * pk.npts)
        rc, _, _ = O.surface_vjp(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v, g)
        assert rel_inf(dc[k], rc) <= G_TOL
