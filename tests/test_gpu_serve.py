"""Serving: requests that share micro-batches and overlap on the GPU get the
same overlays (bit for bit) as when each runs alone, also under a tight
device-memory budget that forces queueing."""
import math
import threading

import numpy as np
import pytest
import torch

import paper_2506_23364_gb300 as awo
from paper_2506_23364_gb300 import inputs
from paper_2506_23364_gb300.serve import OverlayRequest, OverlayServer, latency_summary

pytestmark = pytest.mark.gpu

MU25 = math.tan(math.radians(25.0))


def _requests(n=14):
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(n):
        H, W = int(rng.integers(48, 161)), int(rng.integers(48, 161))
        z = inputs.fbm(max(H, W), 0.8, seed=300 + i, relief=float(rng.uniform(300, 1500)))[:H, :W]
        dem = inputs.quantise_dm(z) if i % 2 == 0 else z.astype(np.float32)
        params = dict(mu=MU25 * float(np.exp(rng.uniform(np.log(0.5), np.log(1.5)))),
                      drag_k=1e-3 * float(np.exp(rng.uniform(np.log(0.5), np.log(1.5)))),
                      traj_per_cell=int(rng.integers(8, 65)), max_steps=int(rng.integers(50, 500)), seed=i)
        reqs.append(OverlayRequest(dem, 10.0, (28.0, 50.0), params, levels=1 + (i % 3)))
    return reqs


def _alone(r: OverlayRequest):
    H, W = r.dem.shape
    ov = awo.Overlay(W, H, r.cell_size, quantised=r.quantised, levels=r.levels)
    ov.load_dem(r.dem)
    ov.run(*r.release_deg, awo.SimParams.make(**r.params), decode_scale=r.decode_scale)
    torch.cuda.synchronize()
    return ov.host_results()


def _serve(reqs, **kw):
    srv = OverlayServer(**kw)
    futs = [None] * len(reqs)

    def submit(idx):
        for i in idx:
            futs[i] = srv.submit(reqs[i])

    ts = [threading.Thread(target=submit, args=(range(k, len(reqs), 2),)) for k in range(2)]
    [t.start() for t in ts]
    [t.join() for t in ts]
    res = [f.result(timeout=120) for f in futs]
    srv.shutdown()
    return srv, res


@pytest.mark.parametrize("kw", [dict(budget_bytes=8 << 30, n_slots=3, max_batch=4),
                                dict(budget_bytes=None, n_slots=2, max_batch=8)])
def test_same_result_alone_and_in_the_mix(kw):
    reqs = _requests()
    alone = [_alone(r) for r in reqs]
    if kw["budget_bytes"] is None:  # room for about two requests at a time
        kw = dict(kw, budget_bytes=2 * max(r.device_bytes() for r in reqs))
    srv, res = _serve(reqs, **kw)
    assert all(r.status == "ok" for r in res), [r.error for r in res]
    assert srv.sched.peak_in_use <= kw["budget_bytes"]
    assert srv.staged_bytes == 0  # every staged DEM went to its flight
    for a, r in zip(alone, res):
        assert len(r.count_lv) == len(a["count_lv"])
        for l in range(len(r.count_lv)):
            assert np.array_equal(r.count_lv[l], a["count_lv"][l]), (r.id, l)
            assert np.array_equal(r.vel_lv[l], a["vel_lv"][l]), (r.id, l)
        assert r.stats == a["stats"]
    assert any(r.batch_size > 1 for r in res) or kw["max_batch"] == 1
    s = latency_summary(res)
    assert s["n"] == len(reqs) and s["p99_ms"] >= s["p50_ms"] > 0


def test_bad_request_fails_alone_on_gpu():
    reqs = _requests(4)
    reqs[1].params = dict(reqs[1].params, persistence=2.0)
    srv, res = _serve(reqs, budget_bytes=8 << 30, n_slots=2, max_batch=4)
    assert [r.status for r in res] == ["ok", "error", "ok", "ok"]


def test_same_result_alone_and_in_the_mix_with_texture_gather_regions():
    """Regions of 2^20 cells and more (footprints by texture gather, as in the
    served 512^2-4096^2 workload) share micro-batches with small ones (loads)
    and still give their single-request overlays bit for bit."""
    reqs = _requests(6)
    rng = np.random.default_rng(11)
    for k, (H, W) in enumerate([(1024, 1024), (1056, 1024)]):
        z = inputs.fbm(max(H, W), 0.8, seed=600 + k, relief=2000.0)[:H, :W]
        params = dict(mu=MU25 * float(np.exp(rng.uniform(np.log(0.5), np.log(1.5)))),
                      drag_k=1e-3 * float(np.exp(rng.uniform(np.log(0.5), np.log(1.5)))),
                      traj_per_cell=8 + 8 * k, max_steps=2000, seed=100 + k)
        reqs.insert(2 + 3 * k, OverlayRequest(inputs.quantise_dm(z), 10.0, (35.0, 45.0), params, levels=2))
    alone = [_alone(r) for r in reqs]
    probe = awo.Overlay(1024, 1024, 10.0, quantised=True, levels=1)
    assert awo.awo_dem_gather_path(probe.h, probe.g) == "texture"
    srv, res = _serve(reqs, budget_bytes=8 << 30, n_slots=2, max_batch=4)
    assert all(r.status == "ok" for r in res), [r.error for r in res]
    for a, r in zip(alone, res):
        for l in range(len(r.count_lv)):
            assert np.array_equal(r.count_lv[l], a["count_lv"][l]), (r.id, l)
            assert np.array_equal(r.vel_lv[l], a["vel_lv"][l]), (r.id, l)
        assert r.stats == a["stats"]
    big = [r for r, q in zip(res, reqs) if q.dem.size >= (1 << 20)]
    assert len(big) == 2 and all(r.stats["n_traj"] > 0 for r in big)
