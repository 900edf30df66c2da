"""Throughput benchmark of the NURBS-Diff hot path on GB300.

Workload (one step): a batch of 256 bicubic NURBS surfaces, 32x32 control nets,
clamped random knots (28 sorted U[0,1] interior knots per direction, every gap
>= 1e-3), weights U[0.5, 2], a 128x128 uniform (u, v) grid; forward evaluation,
MSE against a seeded target surface and the backward pass with gradients for
control points, weights and knots -- all in one libnurbs launch
(nurbs_mse_fwd_bwd).  Metric: surface points per second, forward + backward.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs its own replica of the batch (weak scaling, no
collective on the data path); rank 0 prints one JSON line.

--impl reference times the FP64 CPU oracle (the correctness reference of the
tests) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = {"workload": "256 bicubic NURBS surfaces, 32x32 control nets, random clamped knots, 128x128 grid, "
                        "fwd + MSE + bwd (dP, dw, dU, dV)",
            "batch": 256, "p": 3, "q": 3, "net": 32, "grid": 128}
METRIC = "surface pts/s fwd+bwd FP32"


def run_config(world: int) -> dict:
    """The `config` object of both arms' lines: the workload, how L2 is kept cold
    between timed steps on the GPU arm, and the replica count."""
    return dict(WORKLOAD, l2_flush="256 MiB write before every timed GPU step", parallelism=f"replicas{world}")


def algorithmic_bytes(npts: int, descs) -> int:
    """Bytes the method must move for one fwd+MSE+bwd step.

    Per point: the target read (12 B) and the evaluated point written (12 B).
    Per item: the control net read and its gradient written (16 B per control
    point each), knots read and their gradient written (4 B each), the samples
    read (4 B each) and the item's loss written (4 B).
    """
    b = 24 * npts
    for d in descs:
        nc = int(d["n1"]) * int(d["m1"])
        nk = int(d["n1"] + d["p"] + 1) + int(d["m1"] + d["q"] + 1)
        b += 32 * nc + 8 * nk + 4 * (int(d["nu"]) + int(d["nv"])) + 4
    return b


KERNEL_SOURCES = ("nurbs_tile.cuh", "nurbs_kernel.cuh", "nurbs_basis.cuh", "nurbs_tables.h")


def kernel_sources_sha1() -> str:
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2104_14547_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(tile: str):
    """DRAM bytes (read + write) per launch of the step's kernel from the committed
    ncu capture, or None when the kernel sources or the tile shape differ from
    the ones the counters were taken on."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh)["tiles_kernel_mse_knots_bicubic256"]
    except (OSError, KeyError, ValueError):
        return None
    if rec.get("kernel_sources_sha1") != kernel_sources_sha1() or rec.get("tile") != tile:
        return None
    return rec.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(device, seed: int = 0, with_surfaces: bool = False):
    import torch

    from paper_2104_14547_gb300 import batch, synth
    surfs, targets = synth.bicubic_batch(seed, WORKLOAD["batch"], WORKLOAD["net"], WORKLOAD["grid"])
    pk = batch.pack_surfaces(surfs)
    tk = batch.pack_surfaces(targets)
    kn, ct, pr = batch.to_device(pk, device)
    # the target surface: the forward of an independent control net on the same knots and grid
    tplan = batch.Plan.for_packed(tk, device=device)
    _, tct, _ = batch.to_device(tk, device)
    target = torch.empty((pk.npts, 3), device=device)
    tplan.eval(kn, tct, pr, target)
    torch.cuda.synchronize(device)
    if with_surfaces:
        return pk, kn, ct, pr, target, surfs
    return pk, kn, ct, pr, target


def run_ours(args):
    import torch

    from paper_2104_14547_gb300 import replicas

    # one process per GPU, each with its own seeded shard of independent surfaces
    rk = replicas.init("nccl")
    world, rank, local = rk.world, rk.rank, rk.local
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but {world} rank(s): launch N > 1 under torch.distributed.run")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2104_14547_gb300 import batch, tune

    pk, kn, ct, pr, target, surfs = make_workload(dev, replicas.shard_seed(0, rank), with_surfaces=True)
    npts = pk.npts
    pts = torch.empty((npts, 3), device=dev)
    gc = torch.empty_like(ct)
    gk = torch.empty_like(kn)
    loss = torch.empty(pk.count, device=dev)
    # tile shape from the autotuner (untimed) unless given, then the plan the step runs
    if args.tile:
        best, table = tuple(int(x) for x in args.tile.split(",")), {}
    else:
        best, table = tune.autotune(pk, dict(knots=kn, ctrl=ct, params=pr, target=target, pts=pts, grad_ctrl=gc,
                                             grad_knots=gk, loss=loss), op="mse", device=dev)
    plan = batch.Plan.for_packed(pk, device=dev, warps=best[0], rows=best[1])
    scale = 2.0 / (3.0 * npts)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.mse_fwd_bwd(kn, ct, pr, target, pts, gc, gk, loss, scale)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    st, flags = plan.get_error()
    assert st == 0, (st, flags)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    replicas.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    for k in range(args.steps):
        flush.zero_()                     # L2 flushed before every timed step
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    value = replicas.job_rate(npts * args.steps, float(np.sum(ms)) / 1e3, dev)
    t_ms = replicas.max_over_ranks(float(np.sum(ms)), dev)
    replicas.barrier()
    ms_per_step = t_ms / args.steps

    # roofline of the one kernel of the step (the fused forward+backward tile kernel)
    abytes = algorithmic_bytes(npts, pk.descs)
    achieved = abytes / (ms_per_step / 1e3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    # rows beyond the grid make the same tiles (one tile per surface): key by the effective shape
    traffic = measured_traffic(f"w{best[0]}r{min(best[1], WORKLOAD['grid'])}")

    # end to end through the public API: pinned host inputs in, loss + gradients out
    h_target = target.cpu().pin_memory()
    h_ctrl = ct.cpu().pin_memory()
    h_knots = kn.cpu().pin_memory()
    h_params = pr.cpu().pin_memory()
    h_gc = torch.empty_like(gc, device="cpu").pin_memory()
    h_gk = torch.empty_like(gk, device="cpu").pin_memory()
    h_loss = torch.empty_like(loss, device="cpu").pin_memory()
    bi = sum(t.numel() * t.element_size() for t in (h_target, h_ctrl, h_knots, h_params))
    bo = sum(t.numel() * t.element_size() for t in (h_gc, h_gk, h_loss))

    # pipelined: step k's inputs copy in while step k-1 computes and step k-2's
    # results copy out (two device buffer sets; every step moves bi in, bo out)
    from paper_2104_14547_gb300 import engine
    runner = engine.StreamedSteps(plan, {"knots": h_knots, "ctrl": h_ctrl, "params": h_params, "target": h_target},
                                  {"grad_ctrl": h_gc, "grad_knots": h_gk, "loss": h_loss}, scale, device=dev)
    e0, e1 = runner.run(max(3, args.warmup))
    e1.synchronize()
    torch.cuda.synchronize(dev)
    e0, e1 = runner.run(args.steps)
    e1.synchronize()
    e_ms = e0.elapsed_time(e1)
    e2e_value = replicas.job_rate(npts * args.steps, e_ms / 1e3, dev)

    extras = {}
    want = set(args.extras.split(",")) if args.extras else set()
    xs = max(5, args.steps // 2)
    if rank == 0 and not args.no_extra:
        if "curves" in want:
            extras["curves_fit_step"], extras["curves_eval"] = bench_curves(dev, xs, args.warmup, flush, peak)
        if "derivs" in want:
            extras["tangents_normals"] = bench_derivs(dev, xs, args.warmup, flush, peak, plan, kn, ct, pr, npts,
                                                      pk.descs)
        if "ragged" in want:
            extras["ragged_graph"] = bench_ragged(dev, xs, args.warmup, flush, peak)
        if "offset" in want:
            extras["offset_fit"] = bench_offset(dev, xs, args.warmup, flush, peak)
        if "chamfer" in want:
            extras["chamfer"] = bench_chamfer(dev, xs, args.warmup, flush)
    if rank == 0 and not args.no_extra and ("serve" in want or args.serve):
        # the default run: 20,000 requests at each of the six arrival rates
        extras["serving"] = bench_serve(dev, n_requests=args.serve_requests)

    cpu = parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the outputs of the last timed step, for the oracle leg to compare against
        from paper_2104_14547_gb300 import batch as B
        st, flags = plan.get_error()
        assert st == 0, (st, flags)
        got = {"S": B.unpack_points(pk, pts.cpu().numpy()), "dc": B.unpack_ctrl(pk, gc.cpu().numpy()),
               "dk": B.unpack_knots(pk, gk.cpu().numpy()), "loss": loss.cpu().numpy()}
        cpu, parity = cpu_baseline(surfs, B.unpack_points(pk, target.cpu().numpy()), scale, got,
                                   budget_s=args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "pts/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded, shapes of the paper's fitting workloads)",
            "config": run_config(world),
            "run": {"points_per_step": npts * world, "tile": {"warps": best[0], "rows": best[1]},
                    "autotune_ms": {f"w{w}r{r}": round(v, 4) for (w, r), v in table.items()}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "algorithmic_bytes": abytes,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)" if peaks else "fallback 6.8 TB/s",
                         "kernel": "tiles_kernel<3,3,grad,knots> (nurbs_mse_fwd_bwd)"},
            "e2e": {"value": e2e_value, "unit": "pts/s", "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                    "pipelined": "inputs of step k copy in while step k-1 computes and step k-2's results copy out"},
            "gpu_launches": args.steps * len(set(zip(pk.descs["p"], pk.descs["q"]))),
            "clocks": clk,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if parity is not None:
            line["parity"] = parity
        if extras:
            line["extra"] = extras
        print(json.dumps(line), flush=True)
    replicas.finalize()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover - not Linux
        return os.cpu_count() or 1


def _oracle_step(O, s, T, count):
    """The FP64 oracle on one surface: forward, MSE against T, VJP incl. knots.
    Its C routines release the GIL, so threads run them on all host cores."""
    S = O.surface_eval(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v)
    L, g = O.mse(S, T, count)
    dc, dU, dV = O.surface_vjp(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v, g)
    return S, L, dc, dU, dV


def _rel(a, ref):
    a, ref = np.asarray(a, np.float64), np.asarray(ref, np.float64)
    den = np.abs(ref).max() if ref.size else 0.0
    return float(np.abs(a - ref).max() / den) if den > 0 else float(np.abs(a).max(initial=0.0))


def cpu_baseline(surfs, T, scale, got, budget_s: float = 15.0):
    """The FP64 oracle, as it is, on the host: forward + MSE + VJP of the whole
    workload's surfaces with the step's own target T (an input of the step),
    single-threaded, then on all host cores (a thread per core).  The single-threaded
    pass also yields the oracle's result for every surface, which is compared with
    `got`, the outputs of the last timed GPU step: worst max|dS| / bbox diagonal
    and worst relative gradient error per tensor, over all surfaces."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle as O
    total = sum(s.npts for s in surfs)
    count = 3 * total
    done1, t1, k = 0, 0.0, 0
    worst = {"points_max_abs_over_diag": 0.0, "grad_ctrl_rel": 0.0, "grad_knots_u_rel": 0.0,
             "grad_knots_v_rel": 0.0, "loss_rel": 0.0}
    while k < len(surfs) and t1 < budget_s / 2:
        s = surfs[k]
        Tk = T[k].astype(np.float64)
        ts = time.perf_counter()
        S, L, dc, dU, dV = _oracle_step(O, s, Tk, count)
        t1 += time.perf_counter() - ts
        done1 += s.npts
        xyz = s.ctrl[..., :3].reshape(-1, 3).astype(np.float64)
        diag = float(np.linalg.norm(xyz.max(0) - xyz.min(0)))
        worst["points_max_abs_over_diag"] = max(worst["points_max_abs_over_diag"],
                                                float(np.abs(got["S"][k] - S).max() / diag))
        worst["grad_ctrl_rel"] = max(worst["grad_ctrl_rel"], _rel(got["dc"][k], dc))
        worst["grad_knots_u_rel"] = max(worst["grad_knots_u_rel"], _rel(got["dk"][k][0], dU))
        worst["grad_knots_v_rel"] = max(worst["grad_knots_v_rel"], _rel(got["dk"][k][1], dV))
        ref_loss = L * count
        worst["loss_rel"] = max(worst["loss_rel"], abs(float(got["loss"][k]) - ref_loss) / max(ref_loss, 1e-30))
        k += 1
    parity = dict(worst, surfaces=k, points=done1, bound_points=2e-6, bound_grad=1e-3,
                  within_bound=bool(worst["points_max_abs_over_diag"] <= 2e-6 and
                                    max(worst["grad_ctrl_rel"], worst["grad_knots_u_rel"],
                                        worst["grad_knots_v_rel"]) <= 1e-3),
                  against="FP64 oracle, every sampled surface of the last timed step (same inputs)")
    cores = host_cores()
    pool = ThreadPoolExecutor(max_workers=cores)
    try:
        doneN, tN, passes = 0, 0.0, 0
        idx = list(range(len(surfs)))
        while passes < 1 or tN < budget_s / 2:
            ts = time.perf_counter()
            list(pool.map(lambda j: _oracle_step(O, surfs[j], T[j].astype(np.float64), count), idx))
            tN += time.perf_counter() - ts
            doneN += total
            passes += 1
    finally:
        pool.shutdown()
    cpu = {"value": doneN / tN, "unit": "pts/s", "cores": cores, "kind": "oracle",
           "sample": f"{passes} pass(es) over all {len(surfs)} surfaces ({total} points), fwd + MSE + VJP incl. "
                     f"knots, FP64, {cores} threads (one per host core)",
           "single_core": {"value": done1 / t1, "unit": "pts/s", "cores": 1,
                           "sample": f"{k} of {len(surfs)} surfaces ({done1} points), one thread"}}
    return cpu, parity


def _time_steps(fn, steps, warmup, flush, stream):
    import torch
    for _ in range(warmup):
        flush.zero_()
        fn()
    torch.cuda.synchronize()
    ms = 0.0
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
    return ms / steps


def bench_curves(dev, steps, warmup, flush, peak):
    """4096 cubic 3-D curves, 64 control points, 1024 samples: one fused fit step
    (forward, MSE, backward, Adam on control points and weights) per call, and the
    forward alone (points written, 12 B per sample)."""
    import torch
    from paper_2104_14547_gb300 import batch, synth, tune
    curves, targets = synth.cubic_curve_batch(0, 4096, 64, 1024)
    pk = batch.pack_curves(curves)
    tk = batch.pack_curves(targets)
    kn, ct, pr = batch.to_device(pk, dev)
    _, tct, _ = batch.to_device(tk, dev)
    target = torch.empty((pk.npts, 3), device=dev)
    batch.Plan.for_packed(tk, device=dev).eval(kn, tct, pr, target)
    m, v = torch.zeros_like(ct), torch.zeros_like(ct)
    loss = torch.empty(pk.count, device=dev)
    plan = batch.Plan.for_packed(pk, device=dev, warps=4)
    stream = torch.cuda.current_stream(dev)
    step = [0]

    def fn():
        step[0] += 1
        plan.fit_step(kn, ct, pr, target, m, v, step[0], lr=1e-3, loss_items=loss)

    ms = _time_steps(fn, steps, warmup, flush, stream)
    nctrl = int(pk.descs["n1"].sum())
    abytes = 12 * pk.npts + nctrl * (16 * 2 + 32 * 2) + 4 * (len(pk.knots) + len(pk.params)) + 4 * pk.count
    ach = abytes / (ms / 1e3) / 1e9
    fit = {"workload": "4096 cubic 3-D curves, 64 control points, 1024 samples, fused fit step (fwd + MSE + bwd + Adam)",
           "value": pk.npts / (ms / 1e3), "unit": "curve pts/s", "ms_per_step": ms,
           "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                        "algorithmic_bytes": abytes}}
    pts = torch.empty((pk.npts, 3), device=dev)
    ms = _time_steps(lambda: plan.eval(kn, ct, pr, pts), steps, warmup, flush, stream)
    abytes = 12 * pk.npts + 16 * nctrl + 4 * (len(pk.knots) + len(pk.params))
    ach = abytes / (ms / 1e3) / 1e9
    ev = {"workload": "the same curves, forward only (points written)",
          "value": pk.npts / (ms / 1e3), "unit": "curve pts/s", "ms_per_step": ms,
          "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                       "algorithmic_bytes": abytes}}
    return fit, ev


def bench_derivs(dev, steps, warmup, flush, peak, plan, kn, ct, pr, npts, descs):
    """The bench batch evaluated with tangents and unit normals (points, S_u, S_v,
    normals written: 48 B per point)."""
    import torch
    outs = [torch.empty((npts, 3), device=dev) for _ in range(4)]
    stream = torch.cuda.current_stream(dev)
    ms = _time_steps(lambda: plan.eval_derivs(kn, ct, pr, *outs), steps, warmup, flush, stream)
    abytes = 48 * npts
    for d in descs:
        nc = int(d["n1"]) * int(d["m1"])
        abytes += 16 * nc + 4 * (int(d["n1"] + d["p"] + 1) + int(d["m1"] + d["q"] + 1)) + 4 * (int(d["nu"]) + int(d["nv"]))
    ach = abytes / (ms / 1e3) / 1e9
    return {"workload": "the bench batch, forward with tangents S_u, S_v and unit normals",
            "value": npts / (ms / 1e3), "unit": "surface pts/s", "ms_per_step": ms,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "algorithmic_bytes": abytes}}


def bench_offset(dev, steps, warmup, flush, peak, count=4096):
    """Surface offsetting (Sec. 4) on a batch of bicubic double-curved patches
    (12x12 nets, 20x20 samples): targets from the GPU normals, then fused fit
    steps toward them; time per fit step and the deviation reached."""
    import torch
    from paper_2104_14547_gb300 import offset, synth
    surfs = synth.offset_batch(0, count)
    d = 0.02
    fit = offset.OffsetFit(surfs, d, device=dev)
    stream = torch.cuda.current_stream(dev)
    ms = _time_steps(lambda: fit.step(2e-3), steps, warmup, flush, stream)
    fit.run(max(0, 300 - fit.steps), 2e-3)
    dev_fit = float(fit.deviation().max())
    dev_cp = float(fit.control_point_offset_deviation().max())
    npts = fit.packed.npts
    nctrl = int((fit.packed.descs["n1"] * fit.packed.descs["m1"]).sum())
    abytes = 12 * npts + nctrl * (16 * 2 + 32 * 2) + 4 * (len(fit.packed.knots) + len(fit.packed.params)) + 4 * count
    ach = abytes / (ms / 1e3) / 1e9
    return {"workload": f"{count} bicubic double-curved patches, 12x12 nets, 20x20 samples, offset d = {d}: "
                        "fused fit step toward the offset points",
            "value": npts / (ms / 1e3), "unit": "surface pts/s", "ms_per_step": ms, "tile": list(fit.tile),
            "max_deviation_over_d_after_300_steps": dev_fit / d,
            "control_point_offset_max_deviation_over_d": dev_cp / d,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "algorithmic_bytes": abytes}}


def bench_chamfer(dev, steps, warmup, flush, count=256, grid=64):
    """Chamfer + Hausdorff distances with gradients between the bench surfaces
    evaluated on grid x grid samples and their target surfaces (count pairs of
    grid^2 points each).  ALU-bound: every point meets every point of the other
    set in each direction."""
    import torch
    from paper_2104_14547_gb300 import batch, losses, synth
    surfs, targets = synth.bicubic_batch(0, count, WORKLOAD["net"], grid)
    pk, tk = batch.pack_surfaces(surfs), batch.pack_surfaces(targets)
    kn, ct, pr = batch.to_device(pk, dev)
    _, tct, _ = batch.to_device(tk, dev)
    S = torch.empty((pk.npts, 3), device=dev)
    T = torch.empty((pk.npts, 3), device=dev)
    batch.Plan.for_packed(pk, device=dev).eval(kn, ct, pr, S)
    batch.Plan.for_packed(tk, device=dev).eval(kn, tct, pr, T)
    sizes = [grid * grid] * count
    stream = torch.cuda.current_stream(dev)
    ms = _time_steps(lambda: losses.chamfer(S, sizes, T, sizes), steps, warmup, flush, stream)
    evals = 2 * count * (grid * grid) ** 2          # point-to-point distances, both directions
    ops = 9 * evals                                  # 3 sub, 3 mul, 2 add, 1 compare per distance
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_ops = sms * 128 * 2.07e9                    # FP32 lanes x max SM clock
    return {"workload": f"Chamfer + Hausdorff with gradients, {count} pairs of {grid}x{grid}-point surface samples",
            "value": evals / (ms / 1e3), "unit": "point pairs/s", "ms_per_step": ms,
            "roofline": {"bound": "alu", "achieved": ops / (ms / 1e3) / 1e12, "peak": peak_ops / 1e12,
                         "unit": "TFLOP/s (FP32 non-FMA ops)", "frac": ops / (ms / 1e3) / peak_ops,
                         "peak_source": "152 SMs x 128 FP32 lanes x 2070 MHz"}}


def bench_ragged(dev, steps, warmup, flush, peak, count=1000):
    """1000 surfaces, degrees 2..5, nets 8..64 and grids 32..256 per direction:
    fwd + MSE + bwd through the CUDA-graph engine, against one launch per surface."""
    import torch
    from paper_2104_14547_gb300 import batch, engine, synth
    surfs, targets = synth.ragged_batch(0, count)
    pk = batch.pack_surfaces(surfs)
    tk = batch.pack_surfaces(targets)
    kn, ct, pr = batch.to_device(pk, dev)
    _, tct, _ = batch.to_device(tk, dev)
    tpts = torch.empty((pk.npts, 3), device=dev)
    batch.Plan.for_packed(tk, device=dev).eval(kn, tct, pr, tpts)
    eng = engine.RaggedEngine(surfs, tpts.cpu().numpy(), device=dev)
    eng.capture()
    stream = torch.cuda.current_stream(dev)
    ms = _time_steps(eng.replay, steps, warmup, flush, stream)
    per = engine.PerItemEngine(eng)
    ms_per = _time_steps(per.step, max(2, steps // 5), 1, flush, stream)
    abytes = 0
    for d in pk.descs:
        nc = int(d["n1"]) * int(d["m1"])
        abytes += 24 * int(d["nu"]) * int(d["nv"]) + 32 * nc + 8 * (int(d["n1"] + d["p"] + 1) + int(d["m1"] + d["q"] + 1)) \
            + 4 * (int(d["nu"]) + int(d["nv"])) + 4
    ach = abytes / (ms / 1e3) / 1e9
    return {"workload": f"{count} ragged surfaces (p,q in 2..5, nets 8..64, grids 32..256), fwd + MSE + bwd, "
                        f"{len(eng.groups)} degree groups on parallel streams, one CUDA graph",
            "points": pk.npts, "value": pk.npts / (ms / 1e3), "unit": "surface pts/s", "ms_per_step": ms,
            "per_surface_launches": {"value": pk.npts / (ms_per / 1e3), "ms_per_step": ms_per},
            "speedup_vs_per_surface": ms_per / ms,
            "tiles": {f"p{g['key'][0]}q{g['key'][1]}": list(g["tile"]) for g in eng.groups},
            "step_candidates_ms": {k: round(v, 4) for k, v in eng.step_candidates.items()},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "algorithmic_bytes": abytes}}


def bench_serve(dev, rates=(1000, 2000, 5000, 10000, 20000, 50000), n_requests=20000, seeds=None):
    """Poisson streams of evaluate / fit-step requests on device-resident models
    shaped like the ragged workload; p50/p99 latency and throughput per rate."""
    from paper_2104_14547_gb300 import batch, serve, synth
    import torch
    surfs, targets = synth.ragged_batch(7, 512)
    srv = serve.Server(device=dev, hbm_fraction=0.3, max_wave=256)
    tk = batch.pack_surfaces(targets)
    kn, tct, pr = batch.to_device(tk, dev)
    tpts = torch.empty((tk.npts, 3), device=dev)
    batch.Plan.for_packed(tk, device=dev).eval(kn, tct, pr, tpts)
    T = batch.unpack_points(tk, tpts.cpu().numpy())
    mids = [srv.register(s, t) for s, t in zip(surfs, T)]
    mids = [m for m in mids if m is not None]
    srv.start()
    out = []
    try:
        serve.poisson_run(srv, mids, 500, 2000.0, seed=99)   # warm-up
        for k, rate in enumerate(rates):
            lat, wall, pts, _ = serve.poisson_run(srv, mids, n_requests, float(rate), seed=k)
            out.append({"rate_per_s": rate, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                        "p99_ms": float(np.percentile(lat, 99) * 1e3), "completed_per_s": n_requests / wall,
                        "pts_per_s": pts / wall})
    finally:
        srv.stop()
    return {"workload": f"{n_requests} requests per rate (70% evaluate / 30% fit step) on {len(mids)} resident "
                        "models shaped like the ragged workload", "models": len(mids), "waves": srv.waves,
            "sweep": out}


def run_ragged_group(args):
    """One degree group of the 1000-surface ragged workload, alone: two fused steps
    with the given tile (for a single-kernel profile of a ragged group's kernel)."""
    import torch
    from paper_2104_14547_gb300 import batch, synth
    p, q = (int(x) for x in args.ragged_group.split(","))
    shape = [int(x) for x in (args.tile or "8,128").split(",")]
    w, r, c = (shape + [0])[:3]
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    surfs, targets = synth.ragged_batch(0, 1000)
    pk, tk = batch.pack_surfaces(surfs), batch.pack_surfaces(targets)
    kn, ct, pr = batch.to_device(pk, dev)
    _, tct, _ = batch.to_device(tk, dev)
    T = torch.empty((pk.npts, 3), device=dev)
    batch.Plan.for_packed(tk, device=dev).eval(kn, tct, pr, T)
    sel = np.nonzero((pk.descs["p"] == p) & (pk.descs["q"] == q))[0]
    plan = batch.Plan(pk.kind, pk.descs[sel], device=dev, warps=w, rows=r, ctas_per_sm=c)
    pts, gc, gk = torch.empty_like(T), torch.empty_like(ct), torch.empty_like(kn)
    loss = torch.empty(len(sel), device=dev)
    for _ in range(2):
        plan.mse_fwd_bwd(kn, ct, pr, T, pts, gc, gk, loss, 2.0 / (3 * pk.npts))
    torch.cuda.synchronize(dev)
    d = pk.descs[sel]
    print(json.dumps({"ragged_group": [p, q], "items": int(len(sel)),
                      "points": int((d["nu"].astype(np.int64) * d["nv"]).sum()), "tiles": plan.tiles,
                      "ctas": plan.ctas, "occupancy": list(plan.occupancy("mse_knots")), "tile": [w, r, c],
                      "error": list(plan.get_error())}))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle as O
    from paper_2104_14547_gb300 import synth
    surfs, targets = synth.bicubic_batch(0, WORKLOAD["batch"], WORKLOAD["net"], WORKLOAD["grid"])
    total = WORKLOAD["batch"] * WORKLOAD["grid"] ** 2
    cores = host_cores()
    per_step = cores   # surfaces per step, one per host core: a bounded sample of the workload
    need = min(len(targets), per_step * (args.steps + args.warmup))
    pool = ThreadPoolExecutor(max_workers=cores)
    Ts = list(pool.map(lambda t: O.surface_eval(t.p, t.q, t.U, t.V, t.ctrl, t.u, t.v), targets[:need]))

    def step(k):
        idx = [(k * per_step + j) % len(surfs) for j in range(per_step)]
        list(pool.map(lambda i: _oracle_step(O, surfs[i], Ts[i % len(Ts)], 3 * total), idx))
        return sum(surfs[i].npts for i in idx)

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    pts = 0
    for k in range(args.steps):
        pts += step(args.warmup + k)
    secs = time.perf_counter() - t0
    pool.shutdown()
    value = pts / secs
    line = {"metric": METRIC, "value": value, "unit": "pts/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)", "impl": "reference",
            "config": run_config(int(os.environ.get("WORLD_SIZE", "1"))),
            "run": {"sample_per_step": f"{per_step} surfaces, one thread per host core"},
            "cpu_baseline": {"value": value, "unit": "pts/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} of {WORKLOAD['batch']} surfaces per step, one thread per "
                                       f"host core"},
            "e2e": {"value": value, "unit": "pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-extra", action="store_true", help="skip the extra workloads")
    ap.add_argument("--extras", default="curves,derivs,ragged,offset,chamfer,serve",
                    help="comma-separated extra workloads: curves, derivs, ragged, offset, chamfer, serve "
                         "(Poisson serving sweep, 6 rates)")
    ap.add_argument("--tile", default="", help="fixed tile shape 'warps,rows' instead of the autotuner's "
                    "(with --ragged-group: 'warps,rows[,ctas_per_sm]')")
    ap.add_argument("--ragged-group", default="", help="'p,q': run that degree group of the ragged workload "
                    "alone, two fused steps (for profiling one group's kernel)")
    ap.add_argument("--serve", action="store_true", help="run the serving sweep even when --extras leaves it out")
    ap.add_argument("--serve-requests", type=int, default=20000, help="requests per arrival rate")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.ragged_group:
        run_ragged_group(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
