"""Continuous-batching request server for interactive avalanche overlays.

The paper's workflow recomputes an overlay whenever the user changes a
simulation parameter (Sec. 3: the compute pass re-runs on input or parameter
changes).  A server re-runs it for many users at once:

* requests (a DEM, its cell size, release range, particle parameters and
  mipmap levels) arrive at any time and wait in arrival order;
* the scheduler admits waiting requests as soon as a stream slot is free and
  the device-memory budget has room for their buffers -- requests that arrive
  while others run are admitted into the next micro-batch, they do not wait
  for the running ones to finish;
* a submitted DEM is copied into page-locked host memory on the submitting
  thread (within a host staging budget), so the scheduler thread only issues
  asynchronous copies when the request is admitted;
* an admitted micro-batch (up to ``max_batch`` requests) runs on its own CUDA
  stream: host-to-device copy of the DEMs, terrain stages, ONE batched
  particle launch for all of them (``awo_simulate_batched``), velocity and
  mipmap, device-to-host copy of the overlays -- so micro-batches on
  different slots overlap on the GPU;
* completion is seen through a CUDA event; the request's future then holds
  the overlay (count and velocity rasters of every mipmap level, as arrays
  over the page-locked buffers the device wrote them to: no further copy),
  its statistics and its latency.

A request whose buffers exceed the whole budget is rejected; a request with
invalid parameters fails alone; queued requests can be cancelled.  Because
the batched launch gives every request exactly its single-request result,
a result does not depend on which other requests shared its micro-batch.

``Scheduler`` holds the admission logic and knows nothing about CUDA; the
``GpuExecutor`` runs micro-batches through the library.  Host bookkeeping
only; all arithmetic runs in ``libawo.so``.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# requests and results
# --------------------------------------------------------------------------


@dataclass(eq=False)
class OverlayRequest:
    dem: np.ndarray                   # uint16 decimetres (quantised) or float32 metres
    cell_size: float
    release_deg: tuple[float, float]
    params: dict                      # keyword arguments of SimParams.make
    levels: int = 1
    decode_scale: float = 0.1
    id: int = -1
    t_submit: float = 0.0
    staged: object = field(default=None, repr=False)  # page-locked copy of the DEM, set by the executor
    staged_bytes: int = 0

    @property
    def quantised(self) -> bool:
        return self.dem.dtype == np.uint16

    def device_bytes(self) -> int:
        """Device bytes the request's buffers take (see Overlay + batch workspace)."""
        H, W = self.dem.shape
        n = H * W
        per_cell = (2 if self.quantised else 0) + 4 + 4 + 4 + 4 + 4  # q, h, tan2, count, maxe, vel
        r = int(self.params.get("release_log2", 0))
        if r >= 0:
            entries = n << (2 * r)
        else:
            q = 1 << (-r)
            entries = -(-W // q) * -(-H // q)
        # release list (4 B) and start-record slot (32 B) per release entry, texture mask when r != 0
        per_entry = 4 + 32 + (1 if r else 0)
        lv = 0
        h, w = H, W
        for _ in range(1, self.levels):
            h, w = (h + 1) // 2, (w + 1) // 2
            lv += 8 * h * w
        return n * per_cell + entries * per_entry + lv + (64 << 10)


@dataclass
class OverlayResult:
    id: int
    status: str                       # "ok", "error", "rejected", "cancelled"
    error: str = ""
    count_lv: list = field(default_factory=list)   # uint32 rasters, level 0 first
    vel_lv: list = field(default_factory=list)     # float32 rasters, level 0 first
    stats: dict = field(default_factory=dict)
    batch_size: int = 0
    t_submit: float = 0.0
    t_admit: float = 0.0
    t_done: float = 0.0

    @property
    def latency_s(self) -> float:
        return self.t_done - self.t_submit


# --------------------------------------------------------------------------
# admission logic (no CUDA)
# --------------------------------------------------------------------------


class Scheduler:
    """Arrival-order admission under a slot count and a byte budget.

    ``pick()`` returns the next micro-batch: the longest prefix of the queue
    (at most ``max_batch`` requests) whose device bytes fit in the free
    budget, provided a slot is free.  The head of the queue is never
    overtaken (no starvation of large requests).  Requests larger than the
    whole budget are rejected at submission.
    """

    def __init__(self, budget_bytes: int, n_slots: int, max_batch: int):
        if budget_bytes <= 0 or n_slots < 1 or not 1 <= max_batch <= 128:
            raise ValueError("budget_bytes > 0, n_slots >= 1, 1 <= max_batch <= 128")
        self.budget = int(budget_bytes)
        self.n_slots = int(n_slots)
        self.max_batch = int(max_batch)
        self.queue: deque[OverlayRequest] = deque()
        self.in_use = 0
        self.busy_slots = 0
        self.peak_in_use = 0

    def admissible(self, req: OverlayRequest) -> bool:
        return req.device_bytes() <= self.budget

    def push(self, req: OverlayRequest):
        self.queue.append(req)

    def cancel(self, req_id: int) -> OverlayRequest | None:
        for i, r in enumerate(self.queue):
            if r.id == req_id:
                del self.queue[i]
                return r
        return None

    def pick(self) -> list[OverlayRequest]:
        if self.busy_slots >= self.n_slots or not self.queue:
            return []
        batch, need = [], 0
        for r in self.queue:
            b = r.device_bytes()
            if len(batch) == self.max_batch or self.in_use + need + b > self.budget:
                break
            batch.append(r)
            need += b
        for _ in batch:
            self.queue.popleft()
        if batch:
            self.in_use += need
            self.busy_slots += 1
            self.peak_in_use = max(self.peak_in_use, self.in_use)
        return batch

    def release(self, batch: list[OverlayRequest]):
        self.in_use -= sum(r.device_bytes() for r in batch)
        self.busy_slots -= 1


# --------------------------------------------------------------------------
# GPU executor
# --------------------------------------------------------------------------


class _Flight:
    """One micro-batch in flight on a stream."""

    def __init__(self, reqs, stream, batch, pins, outs, event, t_admit):
        self.reqs, self.stream, self.batch, self.pins = reqs, stream, batch, pins
        self.outs, self.event, self.t_admit = outs, event, t_admit


class GpuExecutor:
    """Launches micro-batches through the library on per-slot CUDA streams."""

    def __init__(self, n_slots: int, device="cuda"):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_slots)]
        self.free = list(range(n_slots))

    def stage(self, req: OverlayRequest):
        """Page-locked host copy of the request's DEM (the source of its
        asynchronous host-to-device copy)."""
        torch = self.torch
        src = np.ascontiguousarray(req.dem)
        if req.quantised:
            src = src.view(np.int16)
        pin = torch.empty(src.shape, dtype=torch.int16 if req.quantised else torch.float32, pin_memory=True)
        pin.numpy()[...] = src
        return pin

    def launch(self, reqs: list[OverlayRequest], t_admit: float) -> _Flight:
        torch = self.torch
        import paper_2506_23364_gb300 as awo

        slot = self.free.pop()
        stream = self.streams[slot]
        params = [awo.SimParams.make(**r.params) for r in reqs]
        with torch.cuda.stream(stream):
            # page-locked DEMs (staged at submission, else here); the flight
            # keeps them until its copies have run
            pins = [r.staged if r.staged is not None else self.stage(r) for r in reqs]
            batch = awo.Batch([r.dem for r in reqs], [r.cell_size for r in reqs], params,
                              [r.release_deg for r in reqs], quantised=[r.quantised for r in reqs],
                              levels=[r.levels for r in reqs], decode_scale=[r.decode_scale for r in reqs],
                              device=self.device, load=False)
            for ov, pin in zip(batch.ovs, pins):
                (ov.q if ov.quantised else ov.h).copy_(pin, non_blocking=True)
            batch.run()
            outs = []
            for ov in batch.ovs:
                cl = [ov.count] + list(ov.count_lv)
                vl = [ov.vel] + list(ov.vel_lv)
                hc = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in cl]
                hv = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in vl]
                for d, h in zip(cl + vl, hc + hv):
                    h.copy_(d, non_blocking=True)
                outs.append((hc, hv))
            hs = torch.empty(batch.stats.shape, dtype=batch.stats.dtype, pin_memory=True)
            hs.copy_(batch.stats, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        fl = _Flight(reqs, stream, batch, pins, (outs, hs), ev, t_admit)
        fl.slot = slot
        return fl

    def done(self, fl: _Flight) -> bool:
        return fl.event.query()

    def collect(self, fl: _Flight) -> list[OverlayResult]:
        import paper_2506_23364_gb300 as awo

        outs, hs = fl.outs
        rows = hs.tolist()
        res = []
        for r, (hc, hv), row in zip(fl.reqs, outs, rows):
            # the result owns the page-locked buffers its arrays view
            res.append(OverlayResult(
                id=r.id, status="ok", count_lv=[h.numpy().view(np.uint32) for h in hc],
                vel_lv=[h.numpy() for h in hv],
                stats={k: int(v) & 0xFFFFFFFFFFFFFFFF for k, v in zip(awo.STATS_FIELDS, row)},
                batch_size=len(fl.reqs), t_submit=r.t_submit, t_admit=fl.t_admit))
        self.free.append(fl.slot)
        return res


# --------------------------------------------------------------------------
# server
# --------------------------------------------------------------------------


class OverlayServer:
    """Submit requests from any thread; one scheduler thread drives the GPU."""

    def __init__(self, budget_bytes: int = 16 << 30, n_slots: int = 4, max_batch: int = 16, device="cuda",
                 executor=None, poll_s: float = 50e-6, host_stage_bytes: int = 4 << 30):
        self.sched = Scheduler(budget_bytes, n_slots, max_batch)
        self.exec = executor if executor is not None else GpuExecutor(n_slots, device)
        self.poll_s = poll_s
        # DEM bytes of queued requests staged in page-locked memory, and its cap
        self.host_stage_bytes = int(host_stage_bytes)
        self.staged_bytes = 0
        self.futures: dict[int, Future] = {}
        self.flights: list = []
        self.lock = threading.Condition()
        self.next_id = 0
        self.stop = False
        self.completed = 0
        self.thread = threading.Thread(target=self._loop, name="awo-serve", daemon=True)
        self.thread.start()

    # ---- client side ---------------------------------------------------
    def submit(self, req: OverlayRequest) -> Future:
        fut: Future = Future()
        self._stage(req)
        with self.lock:
            req.id = self.next_id
            self.next_id += 1
            req.t_submit = time.perf_counter()
            self.futures[req.id] = fut
            err = self._validate(req)
            if err:
                self._unstage(req)
                self._finish(OverlayResult(req.id, "error", err, t_submit=req.t_submit, t_done=time.perf_counter()))
            elif not self.sched.admissible(req):
                self._unstage(req)
                self._finish(OverlayResult(req.id, "rejected", f"needs {req.device_bytes()} device bytes, budget is "
                                           f"{self.sched.budget}", t_submit=req.t_submit, t_done=time.perf_counter()))
            else:
                self.sched.push(req)
                self.lock.notify()
        return fut

    def cancel(self, fut_or_id) -> bool:
        """Cancels a request that is still queued; False once it was admitted or done."""
        with self.lock:
            if isinstance(fut_or_id, int):
                rid = fut_or_id
            else:
                rid = next((k for k, f in self.futures.items() if f is fut_or_id), None)
                if rid is None:
                    return False
            r = self.sched.cancel(rid)
            if r is None:
                return False
            self._unstage(r)
            self._finish(OverlayResult(rid, "cancelled", t_submit=r.t_submit, t_done=time.perf_counter()))
            return True

    def shutdown(self, wait: bool = True):
        with self.lock:
            if wait:
                while (self.sched.queue or self.flights) and not self.stop:
                    self.lock.wait(0.01)
            self.stop = True
            self.lock.notify()
        self.thread.join()

    def _stage(self, req: OverlayRequest):
        """Stages the DEM in page-locked memory on the caller's thread, when the
        executor can and the host staging budget has room; otherwise the
        executor stages it when the request is admitted."""
        stage = getattr(self.exec, "stage", None)
        if stage is None or self._validate(req):
            return
        nbytes = int(req.dem.nbytes)
        with self.lock:
            if self.staged_bytes + nbytes > self.host_stage_bytes:
                return
            self.staged_bytes += nbytes
        try:
            req.staged = stage(req)
            req.staged_bytes = nbytes
        except Exception:  # staging is an optimisation: fall back to staging at admission
            with self.lock:
                self.staged_bytes -= nbytes

    def _unstage(self, req: OverlayRequest):
        """Drops a queued request's staging (from the budget; its buffer goes
        with the request or its flight).  Lock held."""
        self.staged_bytes -= req.staged_bytes
        req.staged_bytes = 0

    # ---- scheduler thread ----------------------------------------------
    @staticmethod
    def _validate(req: OverlayRequest) -> str:
        if req.dem.ndim != 2 or req.dem.dtype not in (np.uint16, np.float32):
            return "dem must be a 2-D uint16 or float32 array"
        lo, hi = req.release_deg
        if not (0.0 <= lo <= hi < 90.0):
            return "release range must satisfy 0 <= lo <= hi < 90"
        if not 1 <= req.levels <= 16:
            return "levels must be in 1..16"
        try:
            import math
            p = dict(req.params)
            P = p.get("persistence", 0.9)
            if not (0.0 <= P <= 1.0) or p.get("randomness", 0.16) < 0 or p.get("mu", 0.47) < 0 or \
                    p.get("drag_k", 0.0) < 0 or not (0 < p.get("step_scale", 1.0) <= 1) or \
                    p.get("drag_k", 0.0) * p.get("step_scale", 1.0) * req.cell_size >= 1 or \
                    not math.isfinite(req.cell_size) or req.cell_size <= 0:
                return "invalid particle parameters"
        except Exception as e:  # malformed parameters
            return f"invalid particle parameters: {e}"
        return ""

    def _finish(self, res: OverlayResult):
        if not res.t_done:
            res.t_done = time.perf_counter()
        fut = self.futures.pop(res.id, None)
        self.completed += 1
        if fut is not None and not fut.done():
            fut.set_result(res)

    def _loop(self):
        try:
            self._run()
        except Exception as e:  # never leave futures hanging
            with self.lock:
                for fl, reqs in self.flights:
                    for r in reqs:
                        self._finish(OverlayResult(r.id, "error", f"server loop failed: {e}", t_submit=r.t_submit))
                self.flights = []
                while self.sched.queue:
                    r = self.sched.queue.popleft()
                    self._finish(OverlayResult(r.id, "error", f"server loop failed: {e}", t_submit=r.t_submit))
                self.stop = True
                self.lock.notify_all()

    def _run(self):
        while True:
            with self.lock:
                if self.stop:
                    return
                # completed micro-batches
                still = []
                for fl, reqs in self.flights:
                    if self.exec.done(fl):
                        for res in self.exec.collect(fl):
                            res.t_done = time.perf_counter()
                            self._finish(res)
                        self.sched.release(reqs)
                    else:
                        still.append((fl, reqs))
                self.flights = still
                # admissions
                while True:
                    batch = self.sched.pick()
                    if not batch:
                        break
                    t_admit = time.perf_counter()
                    try:
                        self.flights.append((self.exec.launch(batch, t_admit), batch))
                    except Exception as e:  # a failing micro-batch fails its own requests only
                        for r in batch:
                            self._finish(OverlayResult(r.id, "error", str(e), t_submit=r.t_submit, t_admit=t_admit))
                        self.sched.release(batch)
                    for r in batch:  # staging now belongs to the flight (or is dropped)
                        self._unstage(r)
                        r.staged = None
                    self.lock.notify_all()
                if not self.flights and not self.sched.queue:
                    self.lock.notify_all()
                    self.lock.wait(0.01)
                    continue
            time.sleep(self.poll_s)


def latency_summary(results: list[OverlayResult]) -> dict:
    lat = np.array([r.latency_s for r in results if r.status == "ok"])
    if lat.size == 0:
        return {"n": 0}
    return {"n": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "max_ms": float(lat.max() * 1e3),
            "mean_ms": float(lat.mean() * 1e3)}
