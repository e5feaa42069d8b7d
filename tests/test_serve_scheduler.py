"""Host-side tests of the serving loop's admission logic with a fake executor
(no GPU): budget and slot limits, arrival order, rejection, cancellation,
failures confined to their micro-batch."""
import threading
import time

import numpy as np
import pytest

from paper_2506_23364_gb300.serve import OverlayRequest, OverlayResult, OverlayServer, Scheduler


class FakeExecutor:
    """Finishes a micro-batch when the test releases it (or immediately)."""

    def __init__(self, auto=True, fail_on=None):
        self.auto = auto
        self.fail_on = fail_on or set()
        self.launched = []
        self.lock = threading.Lock()
        self.inflight_peak = 0
        self.inflight = 0
        self.gate = threading.Event()
        if auto:
            self.gate.set()

    def launch(self, reqs, t_admit):
        if any(r.params.get("tag") in self.fail_on for r in reqs):
            raise RuntimeError("launch failed")
        with self.lock:
            self.launched.append([r.id for r in reqs])
            self.inflight += 1
            self.inflight_peak = max(self.inflight_peak, self.inflight)
        return {"reqs": reqs, "t": t_admit, "at": time.perf_counter()}

    def done(self, fl):
        return self.gate.is_set() and time.perf_counter() - fl["at"] > 0.002

    def collect(self, fl):
        with self.lock:
            self.inflight -= 1
        return [OverlayResult(r.id, "ok", batch_size=len(fl["reqs"]), t_submit=r.t_submit, t_admit=fl["t"])
                for r in fl["reqs"]]


def _req(n=32, tag=None, **kw):
    p = dict(traj_per_cell=4)
    if tag:
        p["tag"] = tag
    p.update(kw)
    return OverlayRequest(np.zeros((n, n), np.float32), 10.0, (30.0, 45.0), p)


def test_budget_and_slots_bound_what_runs():
    one = _req(64).device_bytes()
    ex = FakeExecutor()
    srv = OverlayServer(budget_bytes=2 * one + 10, n_slots=3, max_batch=8, executor=ex)
    futs = [srv.submit(_req(64)) for _ in range(9)]
    res = [f.result(timeout=10) for f in futs]
    srv.shutdown()
    assert all(r.status == "ok" for r in res)
    assert srv.sched.peak_in_use <= 2 * one + 10
    assert all(len(b) <= 2 for b in ex.launched)
    assert sorted(i for b in ex.launched for i in b) == list(range(9))
    assert ex.inflight_peak <= 3


def test_arrival_order_and_max_batch():
    ex = FakeExecutor(auto=False)
    srv = OverlayServer(budget_bytes=1 << 30, n_slots=1, max_batch=3, executor=ex)
    futs = [srv.submit(_req(16)) for _ in range(7)]
    time.sleep(0.05)
    ex.gate.set()
    [f.result(timeout=10) for f in futs]
    srv.shutdown()
    flat = [i for b in ex.launched for i in b]
    assert flat == sorted(flat)
    assert max(len(b) for b in ex.launched) <= 3


def test_oversize_rejected_and_invalid_fails_alone():
    ex = FakeExecutor()
    big = _req(512)
    srv = OverlayServer(budget_bytes=big.device_bytes() - 1, n_slots=2, max_batch=4, executor=ex)
    f_big = srv.submit(big)
    f_bad = srv.submit(_req(16, persistence=1.5))
    f_bad2 = OverlayRequest(np.zeros((8, 8), np.float32), 10.0, (50.0, 40.0), {})
    f_bad2 = srv.submit(f_bad2)
    f_ok = srv.submit(_req(16))
    assert f_big.result(timeout=10).status == "rejected"
    assert f_bad.result(timeout=10).status == "error"
    assert f_bad2.result(timeout=10).status == "error"
    assert f_ok.result(timeout=10).status == "ok"
    srv.shutdown()


def test_cancel_queued_request():
    ex = FakeExecutor(auto=False)
    srv = OverlayServer(budget_bytes=1 << 30, n_slots=1, max_batch=1, executor=ex)
    futs = [srv.submit(_req(16)) for _ in range(4)]
    time.sleep(0.05)
    assert srv.cancel(futs[3]) is True
    ex.gate.set()
    res = [f.result(timeout=10) for f in futs]
    srv.shutdown()
    assert [r.status for r in res] == ["ok", "ok", "ok", "cancelled"]
    assert srv.cancel(0) is False  # already done


def test_failed_launch_fails_its_batch_only():
    ex = FakeExecutor(fail_on={"boom"})
    srv = OverlayServer(budget_bytes=1 << 30, n_slots=1, max_batch=1, executor=ex)
    f1 = srv.submit(_req(16))
    f2 = srv.submit(_req(16, tag="boom"))
    f3 = srv.submit(_req(16))
    assert f1.result(timeout=10).status == "ok"
    r2 = f2.result(timeout=10)
    assert r2.status == "error" and "launch failed" in r2.error
    assert f3.result(timeout=10).status == "ok"
    srv.shutdown()


def test_head_of_queue_not_overtaken():
    s = Scheduler(budget_bytes=_req(64).device_bytes() + _req(16).device_bytes(), n_slots=4, max_batch=8)
    a, b, c = _req(16), _req(64), _req(16)
    for i, r in enumerate((a, b, c)):
        r.id = i
        s.push(r)
    first = s.pick()
    assert [r.id for r in first] == [0, 1]
    assert s.pick() == []  # c waits: budget is full, and it may not overtake
    s.release(first)
    assert [r.id for r in s.pick()] == [2]


def test_scheduler_rejects_bad_configuration():
    with pytest.raises(ValueError):
        Scheduler(0, 1, 1)
    with pytest.raises(ValueError):
        Scheduler(100, 1, 129)


def test_device_bytes_counts_release_texture():
    """The memory estimate grows with the release texture: a start-record
    slot and a list entry per release texel, plus the texture mask."""
    dem = np.zeros((64, 96), np.uint16)
    b0 = OverlayRequest(dem, 10.0, (30.0, 45.0), {}).device_bytes()
    b1 = OverlayRequest(dem, 10.0, (30.0, 45.0), {"release_log2": 1}).device_bytes()
    bm = OverlayRequest(dem, 10.0, (30.0, 45.0), {"release_log2": -1}).device_bytes()
    n = 64 * 96
    assert b1 - b0 == 3 * n * 36 + 4 * n          # 3n more entries, and the 4n-byte mask
    assert b0 - bm == n * 36 - (n // 4) * 37      # a quarter of the entries, with their mask


class StagingExecutor(FakeExecutor):
    """Fake executor that also stages DEMs at submission (as the GPU one does)."""

    def __init__(self, **kw):
        super().__init__(**kw)
        self.staged_ids = []

    def stage(self, req):
        self.staged_ids.append(id(req))
        return object()

    def launch(self, reqs, t_admit):
        fl = super().launch(reqs, t_admit)
        fl["staged"] = [r.staged is not None for r in reqs]
        return fl


def test_host_staging_budget():
    one = _req(64).dem.nbytes
    ex = StagingExecutor(auto=False)
    srv = OverlayServer(budget_bytes=1 << 30, n_slots=1, max_batch=1, executor=ex, host_stage_bytes=3 * one)
    futs = [srv.submit(_req(64)) for _ in range(6)]
    time.sleep(0.05)
    with srv.lock:  # one admitted, five queued: at most three of them staged
        assert 0 < srv.staged_bytes <= 3 * one
        queued_staged = sum(r.staged is not None for r in srv.sched.queue)
        assert queued_staged * one == srv.staged_bytes
    bad = srv.submit(OverlayRequest(np.zeros((8, 8), np.float32), 10.0, (50.0, 40.0), {}))
    assert bad.result(timeout=5).status == "error"
    ex.gate.set()
    res = [f.result(timeout=10) for f in futs]
    srv.shutdown()
    assert all(r.status == "ok" for r in res)
    assert srv.staged_bytes == 0
    assert len(ex.staged_ids) >= 3
