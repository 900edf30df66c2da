"""Continuous-batching server for surface evaluation and fit-step requests.

Models (NURBS surfaces with a fitting target) live on the device in an arena:
knots, control nets, samples, targets and Adam moments.  The arena is sized from
the free HBM at start-up; registering a model succeeds only while it has room
(admission by free HBM).  Clients submit requests that name a model:

* ``eval``  -- evaluate the model's current surface on its grid; the points come back;
* ``fit``   -- one fused step (forward, MSE against the stored target, backward,
  Adam update of the control net in place); the loss comes back.  The loss of a
  fit request is the mean over its own model's points (Sec. 4, Eq. 12): each
  item of a fit wave carries its own gradient scale, so a model's trajectory is
  the same whichever requests share its waves;
* ``checkpoint`` / ``restore`` -- barriers in arrival order: the scheduler lets
  the waves in flight finish, then copies every model's control net, Adam moments
  and step count to host memory (``checkpoint``, the result) or back
  (``restore``, ``Request.payload`` = a checkpoint), so that a fit after a
  restore continues bit for bit where the checkpoint left off.

A request can be cancelled (``Request.cancel``) until a wave admits it; it then
completes at once with ``error == "cancelled"`` and never reaches the GPU.  Once
admitted it runs to completion.

A scheduler thread forms waves from the pending requests in arrival order.  A
wave holds at most one request per model and as many evaluations as the output
region has room for; requests that do not fit wait for the next wave.  Each wave
is one libnurbs plan per kind (eval / fit) launched on its own stream; up to two
waves are in flight at once, so requests that arrive while a wave runs start on
the device before it finishes.  A finished wave's evaluation results are copied
into the requests' host arrays by the scheduler itself when the wave is small,
and by a small pool of copy threads when it is large (under heavy load the
copies, not the scheduling, bound the served request rate; handing a small wave
to another thread costs more latency than its copy), while the scheduler forms
and launches the next waves.  The plans bind to workspaces kept in a pool (one
per wave slot and kind, grown when a wave needs more), so forming a wave
allocates no device memory.  Every request records its latency (submit to result
on the host).
"""
from __future__ import annotations

import collections
import concurrent.futures
import os
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib, batch


def copy_chunks(sizes, workers: int):
    """Bounds [0, b1, ..., len(sizes)] that cut a wave's evaluations into at most
    `workers` contiguous chunks of about equal total size (in points), none empty."""
    n = len(sizes)
    if n == 0:
        return [0]
    k = max(1, min(workers, n))
    cum = np.cumsum(np.asarray(sizes, dtype=np.int64))
    cuts = np.searchsorted(cum, cum[-1] * np.arange(1, k) / k) + 1
    return [0, *sorted(set(int(c) for c in cuts if 0 < c < n)), n]


class RangeAllocator:
    """First-fit free list over [0, size) (units: elements)."""

    def __init__(self, size: int):
        self.size = size
        self.free = [(0, size)]

    def alloc(self, n: int, align: int = 1):
        for k, (o, ln) in enumerate(self.free):
            a = (o + align - 1) // align * align
            if a + n <= o + ln:
                rest = []
                if a > o:
                    rest.append((o, a - o))
                if a + n < o + ln:
                    rest.append((a + n, o + ln - a - n))
                self.free[k: k + 1] = rest
                return a
        return None

    def release(self, off: int, n: int):
        self.free.append((off, n))
        self.free.sort()
        merged = []
        for o, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((o, ln))
        self.free = merged

    @property
    def available(self) -> int:
        return sum(ln for _, ln in self.free)


@dataclass
class Model:
    mid: int
    p: int
    q: int
    n1: int
    m1: int
    nu: int
    nv: int
    knot_u: int
    knot_v: int
    ctrl: int
    param_u: int
    param_v: int
    target: int
    steps: int = 0


@dataclass
class Request:
    kind: str                 # "eval", "fit", "checkpoint" or "restore"
    model: int = -1
    t_submit: float = 0.0
    t_done: float = 0.0
    result: object = None
    error: str | None = None  # set when the server failed (or cancelled) the request
    payload: object = None    # "restore": the checkpoint to put back
    out: np.ndarray | None = None   # "eval": float32 array of the model's nu*nv*3 floats to fill (else allocated)
    cancelled: bool = False
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit

    def cancel(self):
        """Withdraw the request; takes effect if no wave has admitted it yet."""
        self.cancelled = True


class Server:
    def __init__(self, device="cuda", hbm_fraction=0.25, max_wave=256, out_points=1 << 24, lr=1e-3,
                 warps=4, rows=32, max_models=1 << 14, copy_workers=None, inline_copy_points=1 << 18):
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self._inflight_requests = []
        free, _ = torch.cuda.mem_get_info(self.device)
        budget = int(free * hbm_fraction)
        # arena split by element size: ctrl/m/v 48 B per control point, targets 12 B per point,
        # knots/samples 4 B each; sized for grids ~ (8 x net)^2
        unit = 48 * 64 + 12 * 4096 + 4 * 200
        n_units = max(64, budget // unit)
        self.n_ctrl, self.n_pts, self.n_scalar = 64 * n_units, 4096 * n_units, 200 * n_units
        self.ctrl = torch.zeros((self.n_ctrl, 4), device=self.device)
        self.adam_m = torch.zeros_like(self.ctrl)
        self.adam_v = torch.zeros_like(self.ctrl)
        self.scalars = torch.zeros(self.n_scalar, device=self.device)   # knots and samples
        self.target = torch.zeros((self.n_pts, 3), device=self.device)
        self.out = [torch.zeros((out_points, 3), device=self.device) for _ in range(2)]
        self.host_out = [torch.empty((out_points, 3), pin_memory=True) for _ in range(2)]
        self.host_loss = [torch.empty(max_wave, pin_memory=True) for _ in range(2)]
        self.loss = [torch.zeros(max_wave, device=self.device) for _ in range(2)]
        self.alloc_ctrl = RangeAllocator(self.n_ctrl)
        self.alloc_pts = RangeAllocator(self.n_pts)
        self.alloc_scalar = RangeAllocator(self.n_scalar)
        self.models: dict[int, Model] = {}
        # the models' descriptor fields as one int64 table (row = model id), for building a
        # wave's descriptors with array operations: p q n1 m1 nu nv knot_u knot_v ctrl
        # param_u param_v target steps
        self._mt = np.zeros((0, 13), np.int64)
        self.max_wave = max_wave
        self.out_points = out_points
        self.lr = lr
        self.tile = dict(warps=warps, rows=rows)
        self.streams = [(torch.cuda.Stream(self.device), torch.cuda.Stream(self.device)) for _ in range(2)]
        # plan workspaces, one per (wave slot, kind): reused by every wave on that slot
        self.ws_pool = {(slot, kind): torch.zeros(1 << 20, dtype=torch.uint8, device=self.device)
                        for slot in range(2) for kind in ("eval", "fit")}
        self.queue: collections.deque[Request] = collections.deque()
        self.cv = threading.Condition()
        self.running = False
        self.thread = None
        self.waves = 0
        self.points_done = 0
        self.failure: str | None = None
        # result copies of finished waves: a thread pool, and per wave slot the copies
        # still reading that slot's pinned host buffer
        self.copy_workers = copy_workers or max(1, min(8, os.cpu_count() or 1))
        self.inline_copy_points = inline_copy_points   # waves with fewer evaluated points copy inline
        self._copy_pool = None
        self._copies = [[], []]

    # ------------------------------------------------------------ models
    def register(self, surface, target_pts: np.ndarray) -> int | None:
        """Place a model in the arena; None when it does not fit (admission by free HBM)."""
        s = surface
        n1, m1 = s.ctrl.shape[0], s.ctrl.shape[1]
        nk, ns, npts = len(s.U) + len(s.V), len(s.u) + len(s.v), len(s.u) * len(s.v)
        c = self.alloc_ctrl.alloc(n1 * m1)
        if c is None:
            return None
        t = self.alloc_pts.alloc(npts)
        if t is None:
            self.alloc_ctrl.release(c, n1 * m1)
            return None
        k = self.alloc_scalar.alloc(nk + ns)
        if k is None:
            self.alloc_ctrl.release(c, n1 * m1)
            self.alloc_pts.release(t, npts)
            return None
        dev = self.device
        self.ctrl[c: c + n1 * m1] = torch.from_numpy(np.asarray(s.ctrl, np.float32).reshape(-1, 4)).to(dev)
        self.adam_m[c: c + n1 * m1] = 0
        self.adam_v[c: c + n1 * m1] = 0
        self.scalars[k: k + nk + ns] = torch.from_numpy(
            np.concatenate([s.U, s.V, s.u, s.v]).astype(np.float32)).to(dev)
        self.target[t: t + npts] = torch.from_numpy(np.asarray(target_pts, np.float32).reshape(-1, 3)).to(dev)
        mid = len(self.models)
        self.models[mid] = Model(mid, s.p, s.q, n1, m1, len(s.u), len(s.v), k, k + len(s.U), c,
                                 k + nk, k + nk + len(s.u), t)
        row = np.array([[s.p, s.q, n1, m1, len(s.u), len(s.v), k, k + len(s.U), c, k + nk, k + nk + len(s.u), t, 0]],
                       np.int64)
        self._mt = np.concatenate([self._mt, row])
        return mid

    # ------------------------------------------------------------ requests
    def submit(self, req: Request) -> Request:
        req.t_submit = time.perf_counter()
        if self.failure is not None:
            req.error = self.failure
            req.done.set()
            return req
        with self.cv:
            self.queue.append(req)
            self.cv.notify()
        return req

    def start(self):
        self.running = True
        self._copy_pool = concurrent.futures.ThreadPoolExecutor(max_workers=self.copy_workers,
                                                                thread_name_prefix="nurbs-serve-copy")
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def stop(self):
        with self.cv:
            self.running = False
            self.cv.notify()
        if self.thread is not None:
            self.thread.join()
        if self._copy_pool is not None:
            self._copy_pool.shutdown(wait=True)
            self._copy_pool = None

    def _form_wave(self, busy: set):
        """Pending requests admitted into one wave (arrival order, one per model,
        evaluation outputs while the output region has room).  Stops at a
        checkpoint or restore barrier, which runs on its own."""
        evals, fits, out_used, keep = [], [], 0, collections.deque()
        while self.queue and len(evals) + len(fits) < self.max_wave:
            r = self.queue.popleft()
            if r.cancelled:
                self._finish_cancelled(r)
                continue
            if r.kind in ("checkpoint", "restore"):
                keep.append(r)
                break
            m = self.models[r.model]
            if r.model in busy:
                keep.append(r)
                continue
            if r.kind == "eval":
                n = m.nu * m.nv
                if out_used + n > self.out_points:
                    keep.append(r)
                    break
                evals.append((r, out_used))
                out_used += n
            else:
                fits.append(r)
            busy.add(r.model)
        while keep:
            self.queue.appendleft(keep.pop())
        return evals, fits

    @staticmethod
    def _finish_cancelled(r: Request):
        r.error = "cancelled"
        r.t_done = time.perf_counter()
        r.done.set()

    def _descs(self, entries, fit: bool):
        mids = np.fromiter(((e if fit else e[0]).model for e in entries), np.int64, len(entries))
        t = self._mt[mids]
        d = np.zeros(len(entries), batch.DESC_DTYPE)
        for k, name in enumerate(("p", "q", "n1", "m1", "nu", "nv")):
            d[name] = t[:, k]
        for k, name in enumerate(("knot_u", "knot_v", "ctrl", "param_u", "param_v"), start=6):
            d[name] = t[:, k]
        if fit:
            d["adam_step"] = t[:, 12] + 1
            # a fit item's loss is the mean over its own points: grad_scale 2 / (3 nu nv)
            d["grad_scale"] = (2.0 / (3.0 * np.maximum(t[:, 4] * t[:, 5], 1))).astype(np.float32)
            d["pts"] = t[:, 11]
        else:
            d["pts"] = np.fromiter((off for _, off in entries), np.int64, len(entries))
        return d

    def _plan(self, slot, kind, descs):
        """A plan bound to the pooled workspace of (slot, kind), grown if it is too small."""
        plan = None
        key = (slot, kind)
        try:
            plan = batch.Plan(_lib.KIND_SURFACE, descs, device=self.device, workspace=self.ws_pool[key],
                              **self.tile)
        except ValueError:
            probe = batch.Plan(_lib.KIND_SURFACE, descs, device=self.device, workspace=None, **self.tile)
            self.ws_pool[key] = probe.workspace
            plan = probe
        return plan

    def _launch(self, slot, evals, fits):
        se, sf = self.streams[slot]
        main = torch.cuda.current_stream(self.device)
        # the copies of the slot's previous wave must be done reading its pinned buffer
        # before this wave's results are copied into it
        for f in self._copies[slot]:
            f.result()
        self._copies[slot] = []
        # plans first: their tables are uploaded into the pooled workspaces on the current stream
        pe = self._plan(slot, "eval", self._descs(evals, False)) if evals else None
        pf = self._plan(slot, "fit", self._descs(fits, True)) if fits else None
        se.wait_stream(main)
        sf.wait_stream(main)
        plans = []
        n_out = 0
        if evals:
            pe.eval(self.scalars, self.ctrl, self.scalars, self.out[slot], stream=se)
            n_out = sum(self.models[r.model].nu * self.models[r.model].nv for r, _ in evals)
            with torch.cuda.stream(se):
                self.host_out[slot][:n_out].copy_(self.out[slot][:n_out], non_blocking=True)
            plans.append(pe)
        if fits:
            # every item carries its own grad_scale and Adam step (see _descs)
            pf.fit_step(self.scalars, self.ctrl, self.scalars, self.target, self.adam_m, self.adam_v, 1,
                        lr=self.lr, loss_items=self.loss[slot], stream=sf)
            with torch.cuda.stream(sf):
                self.host_loss[slot][: len(fits)].copy_(self.loss[slot][: len(fits)], non_blocking=True)
            plans.append(pf)
        ev = torch.cuda.Event()
        ev.record(se)
        ev2 = torch.cuda.Event()
        ev2.record(sf)
        return dict(slot=slot, evals=evals, fits=fits, plans=plans, events=(ev, ev2), n_out=n_out)

    @staticmethod
    def _deliver(ho, entries, shapes):
        """Copy finished evaluations out of a wave's pinned buffer into their requests
        and complete them (runs on a copy thread)."""
        for (r, off), (nu, nv) in zip(entries, shapes):
            try:
                n = nu * nv
                src = ho[off: off + n]
                if r.out is not None:        # the caller's own buffer: no allocation here
                    np.copyto(r.out.reshape(-1, 3)[:n], src)
                    r.result = r.out
                else:
                    r.result = src.reshape(nu, nv, 3).copy()
            except Exception as exc:  # the request fails, the server goes on
                r.error = f"result copy failed: {exc!r}"
            r.t_done = time.perf_counter()
            r.done.set()

    def _complete(self, w, busy: set):
        for e in w["events"]:
            e.synchronize()
        now = time.perf_counter()
        ho = self.host_out[w["slot"]].numpy()
        evals = w["evals"]
        shapes = [(self.models[r.model].nu, self.models[r.model].nv) for r, _ in evals]
        for r, _ in evals:
            busy.discard(r.model)        # the device side of the wave is done
        npts = sum(nu * nv for nu, nv in shapes)
        self.points_done += npts
        if evals and npts <= self.inline_copy_points:
            self._deliver(ho, evals, shapes)
        elif evals:
            bounds = copy_chunks([nu * nv for nu, nv in shapes], self.copy_workers)
            for a, b in zip(bounds[:-1], bounds[1:]):
                self._copies[w["slot"]].append(self._copy_pool.submit(self._deliver, ho, evals[a:b], shapes[a:b]))
        hl = self.host_loss[w["slot"]].numpy()
        for k, r in enumerate(w["fits"]):
            m = self.models[r.model]
            m.steps += 1
            self._mt[r.model, 12] = m.steps
            r.result = float(hl[k]) / (3.0 * m.nu * m.nv)
            self.points_done += m.nu * m.nv
        for r in w["fits"]:
            busy.discard(r.model)
            r.t_done = now
            r.done.set()

    def _loop(self):
        try:
            self._serve()
        except BaseException as exc:  # fail every waiting request instead of leaving it hanging
            import traceback
            self.failure = "".join(traceback.format_exception(exc))
            with self.cv:
                pending = list(self.queue)
                self.queue.clear()
                self.running = False
            for r in pending + self._inflight_requests:
                if not r.done.is_set():
                    r.error = self.failure
                    r.done.set()

    # ------------------------------------------------------------ checkpoint / restore
    def _checkpoint(self) -> dict:
        """Host copies of every model's control net, Adam moments and step count
        (run by the scheduler with no wave in flight)."""
        ck = {"models": {}}
        for mid, m in self.models.items():
            n = m.n1 * m.m1
            ck["models"][mid] = dict(ctrl=self.ctrl[m.ctrl: m.ctrl + n].cpu(),
                                     adam_m=self.adam_m[m.ctrl: m.ctrl + n].cpu(),
                                     adam_v=self.adam_v[m.ctrl: m.ctrl + n].cpu(), steps=m.steps)
        return ck

    def _restore(self, ck: dict):
        for mid, st in ck["models"].items():
            m = self.models[mid]
            n = m.n1 * m.m1
            if st["ctrl"].shape[0] != n:
                raise ValueError(f"checkpoint of model {mid} does not match its control net")
            self.ctrl[m.ctrl: m.ctrl + n] = st["ctrl"].to(self.device)
            self.adam_m[m.ctrl: m.ctrl + n] = st["adam_m"].to(self.device)
            self.adam_v[m.ctrl: m.ctrl + n] = st["adam_v"].to(self.device)
            m.steps = int(st["steps"])
            self._mt[mid, 12] = m.steps
        torch.cuda.synchronize(self.device)

    def checkpoint(self, timeout: float = 60.0) -> dict:
        """Snapshot of every model's device-resident state, taken after the
        requests submitted before this call (a barrier in arrival order)."""
        r = self.submit(Request("checkpoint"))
        if not r.done.wait(timeout) or r.error is not None:
            raise RuntimeError(f"checkpoint failed: {r.error or 'timeout'}")
        return r.result

    def restore(self, ck: dict, timeout: float = 60.0):
        """Put a checkpoint back (a barrier in arrival order, like checkpoint)."""
        r = self.submit(Request("restore", payload=ck))
        if not r.done.wait(timeout) or r.error is not None:
            raise RuntimeError(f"restore failed: {r.error or 'timeout'}")

    def _serve(self):
        torch.cuda.set_device(self.device)
        inflight: collections.deque = collections.deque()
        self._inflight_requests = []
        busy: set = set()
        slot = 0
        while True:
            barrier = None
            with self.cv:
                while self.running and not self.queue and not inflight:
                    self.cv.wait(timeout=0.05)
                if not self.running and not self.queue and not inflight:
                    return
                wave = self._form_wave(busy) if len(inflight) < 2 and self.queue else ([], [])
                if not (wave[0] or wave[1]) and not inflight and self.queue and \
                        self.queue[0].kind in ("checkpoint", "restore"):
                    barrier = self.queue.popleft()
            if barrier is not None:
                # every earlier wave has finished: the arena holds their results
                if barrier.cancelled:
                    self._finish_cancelled(barrier)
                    continue
                if barrier.kind == "checkpoint":
                    barrier.result = self._checkpoint()
                else:
                    self._restore(barrier.payload)
                barrier.t_done = time.perf_counter()
                barrier.done.set()
                continue
            evals, fits = wave
            if evals or fits:
                self._inflight_requests = [r for r, _ in evals] + list(fits) + \
                    [r for r in self._inflight_requests if not r.done.is_set()]
                inflight.append(self._launch(slot, evals, fits))
                slot ^= 1
                self.waves += 1
            elif inflight:
                self._complete(inflight.popleft(), busy)
                continue
            # retire finished waves without blocking the next launch
            while inflight and (len(inflight) == 2 or all(e.query() for e in inflight[0]["events"])):
                self._complete(inflight.popleft(), busy)


def poisson_run(server: Server, model_ids, n_requests: int, rate: float, eval_frac: float = 0.7, seed: int = 0):
    """Submit n_requests with exponential inter-arrival times at `rate` per second;
    returns (latencies in seconds, wall seconds, points processed, requests).

    A load generator, not a client that keeps results: every evaluation of a model
    fills that model's one output array (overwritten by its later evaluations), and
    Python's cyclic garbage collector is paused during the run, so that host-side
    allocation and collection pauses do not show up as serving latency."""
    import gc

    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    kinds = rng.random(n_requests) < eval_frac
    mids = rng.choice(model_ids, size=n_requests)
    outs = {int(m): np.empty(server.models[int(m)].nu * server.models[int(m)].nv * 3, np.float32)
            for m in set(mids.tolist())}
    reqs = []
    gc_was = gc.isenabled()
    gc.collect()
    gc.disable()
    try:
        p0 = server.points_done
        t0 = time.perf_counter()
        t_next = t0
        for k in range(n_requests):
            t_next += gaps[k]
            while True:
                dt = t_next - time.perf_counter()
                if dt <= 0:
                    break
                time.sleep(min(dt, 0.001) if dt > 2e-4 else 0)
            m = int(mids[k])
            reqs.append(server.submit(Request("eval", m, out=outs[m]) if kinds[k] else Request("fit", m)))
        for r in reqs:
            if not r.done.wait(timeout=120.0) or r.error is not None:
                raise RuntimeError(f"request not served: {r.error or 'timeout'}")
        wall = time.perf_counter() - t0
    finally:
        if gc_was:
            gc.enable()
    return np.array([r.latency for r in reqs]), wall, server.points_done - p0, reqs
