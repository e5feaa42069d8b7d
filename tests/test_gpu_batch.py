"""Batched particle launch: every region's rasters and statistics equal those
of the single-region call (and hence the oracle's), for every launch shape
of the autotuner's search space, with shared or per-region seeds, eagerly and
replayed from a CUDA graph."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2506_23364_gb300 as awo
from paper_2506_23364_gb300 import inputs

pytestmark = pytest.mark.gpu

MU25 = math.tan(math.radians(25.0))


def _regions(seed_mode="mixed"):
    rng = np.random.default_rng(42)
    dems, params, rel = [], [], []
    shapes = [(96, 130), (64, 64), (150, 97), (33, 200), (128, 128), (80, 81)]
    for i, (H, W) in enumerate(shapes):
        z = inputs.fbm(max(H, W), 0.8, seed=200 + i, relief=float(rng.uniform(400, 1200)))[:H, :W]
        dems.append(z.astype(np.float32))
        p = awo.SimParams.make(mu=MU25 * float(np.exp(rng.uniform(np.log(0.5), np.log(1.5)))),
                               drag_k=1e-3 * float(np.exp(rng.uniform(np.log(0.5), np.log(1.5)))),
                               persistence=float(rng.uniform(0.5, 0.95)), randomness=float(rng.uniform(0.05, 0.4)),
                               traj_per_cell=int(rng.choice([1, 7, 32, 33, 100])), max_steps=int(rng.integers(5, 400)),
                               seed=(i * 7919 if seed_mode == "mixed" else 5))
        params.append(p)
        rel.append((25.0, 50.0))
    return dems, params, rel


def _plain(dem, p, lo, hi):
    H, W = dem.shape
    ov = awo.Overlay(W, H, 10.0, quantised=False, levels=1)
    ov.load_dem(dem)
    ov.run(lo, hi, p)
    torch.cuda.synchronize()
    return ov.host_results()


def _check_against_plain(b: awo.Batch, dems, params, rel):
    st = b.stats_list()
    for i, (dem, p, (lo, hi)) in enumerate(zip(dems, params, rel)):
        ref = _plain(dem, p, lo, hi)
        got = b.results(i)
        assert np.array_equal(got["cells"], ref["cells"]), i
        assert np.array_equal(got["count"], ref["count"]), i
        assert np.array_equal(got["maxe"], ref["maxe"]), i
        assert np.array_equal(got["vel"], ref["vel"]), i
        assert st[i] == ref["stats"], (i, st[i], ref["stats"])


@pytest.mark.parametrize("seed_mode", ["mixed", "shared"])
def test_batched_equals_plain(seed_mode):
    dems, params, rel = _regions(seed_mode)
    b = awo.Batch(dems, 10.0, params, rel, quantised=False)
    b.run()
    torch.cuda.synchronize()
    _check_against_plain(b, dems, params, rel)


def test_batched_matches_oracle_directly():
    dems, params, rel = _regions()
    b = awo.Batch(dems[:3], 10.0, params[:3], rel[:3], quantised=False)
    b.run()
    torch.cuda.synchronize()
    for i in range(3):
        p = params[i]
        op = oracle.SimParams(mu=p.mu, drag_k=p.drag_k, persistence=p.persistence, randomness=p.randomness,
                              step_scale=p.step_scale, gravity=p.gravity, traj_per_cell=p.traj_per_cell,
                              max_steps=p.max_steps, seed=p.seed)
        ref = oracle.overlay(dems[i], 10.0, *rel[i], op)
        got = b.results(i)
        assert np.array_equal(got["count"], ref["count"]) and np.array_equal(got["vel"], ref["vel"]), i


def test_every_tuning_gives_the_same_rasters():
    dems, params, rel = _regions()
    b = awo.Batch(dems, 10.0, params, rel, quantised=False)
    b.run()
    torch.cuda.synchronize()
    base = [b.results(i) for i in range(b.n)]
    base_stats = b.stats_list()
    for rf in (awo.REFILL_LANE, awo.REFILL_WARP):
        for th in (64, 128, 256):
            for gp in (0, 32, 100, 256, 1024, 4096):
                b.tuning = awo.Tuning(th, gp, rf, 0)
                b.run()
                torch.cuda.synchronize()
                for i in range(b.n):
                    got = b.results(i)
                    assert np.array_equal(got["count"], base[i]["count"]), (rf, th, gp, i)
                    assert np.array_equal(got["maxe"], base[i]["maxe"]), (rf, th, gp, i)
                assert b.stats_list() == base_stats


def test_tuner_and_graph_replay():
    dems, params, rel = _regions()
    b = awo.Batch(dems, 10.0, params, rel, quantised=False)
    best, ms = b.tune()
    assert best.threads_per_block in (64, 128, 256) and best.refill in (0, 1) and ms > 0
    torch.cuda.synchronize()
    tuned = [b.results(i) for i in range(b.n)]  # the tuner leaves the batch's result in the rasters
    b.capture()
    for _ in range(2):
        for ov in b.ovs:
            ov.count.fill_(7)  # scribble: the replay must clear and recompute
        b.replay()
        torch.cuda.synchronize()
    _check_against_plain(b, dems, params, rel)
    for i in range(b.n):
        assert np.array_equal(b.results(i)["count"], tuned[i]["count"])


def test_batched_edge_requests():
    z = inputs.fbm(64, 0.8, seed=9, relief=900.0).astype(np.float32)
    flat = np.full((20, 30), 100.0, np.float32)
    gentle = inputs.plane(50, 40, 10.0, math.tan(math.radians(20.0)))
    dems = [z, flat, z, z, gentle]
    params = [awo.SimParams.make(traj_per_cell=16, max_steps=50), awo.SimParams.make(traj_per_cell=8),
              awo.SimParams.make(traj_per_cell=0), awo.SimParams.make(traj_per_cell=5, max_steps=0),
              awo.SimParams.make(traj_per_cell=3, max_steps=1)]
    rel = [(30.0, 45.0), (0.0, 10.0), (30.0, 45.0), (30.0, 45.0), (80.0, 85.0)]  # last: no release cell
    b = awo.Batch(dems, 10.0, params, rel, quantised=False)
    b.run()
    torch.cuda.synchronize()
    _check_against_plain(b, dems, params, rel)
    st = b.stats_list()
    assert st[2]["n_traj"] == 0 and st[4]["n_traj"] == 0
    assert st[3]["n_capped"] == st[3]["n_traj"] > 0


def test_single_request_batch_equals_awo_simulate_on_tiny():
    w = inputs.tiny()
    p = awo.SimParams.make(traj_per_cell=16, max_steps=1000)
    b = awo.Batch([w.dem_f32], 10.0, [p], [(30.0, 45.0)], quantised=False)
    b.run()
    torch.cuda.synchronize()
    _check_against_plain(b, [w.dem_f32], [p], [(30.0, 45.0)])


# ----------------------------------------------------------------------------
# Regions of 2^20 cells and more: the batched kernel gathers their footprints
# through per-request texture views (when the DEM buffer's address and row
# pitch meet the texture alignment), in the same launch as regions that take
# loads.  The 512^2-4096^2 batched and served workloads run this path.
# ----------------------------------------------------------------------------
BIG_SPECS = [  # (H, W, uint16 dm storage, expected footprint path)
    (1040, 1024, False, "texture"),  # 4096-byte rows
    (1024, 1280, True, "texture"),   # uint16 dm, decoded into an aligned FP32 buffer
    (1024, 1025, False, "loads"),    # 4100-byte rows: off the texture pitch alignment
    (96, 130, False, "loads"),       # under 2^20 cells
    (150, 97, True, "loads"),
    (64, 64, False, "loads"),
]


def _big_regions():
    rng = np.random.default_rng(77)
    dems, params, rel, qz = [], [], [], []
    for i, (H, W, q, _) in enumerate(BIG_SPECS):
        z = inputs.fbm(max(H, W), 0.8, seed=500 + i, relief=float(rng.uniform(1500, 2500)))[:H, :W]
        dems.append(inputs.quantise_dm(z) if q else z.astype(np.float32))
        qz.append(q)
        params.append(awo.SimParams.make(
            mu=MU25 * float(np.exp(rng.uniform(np.log(0.5), np.log(1.5)))),
            drag_k=1e-3 * float(np.exp(rng.uniform(np.log(0.5), np.log(1.5)))),
            persistence=float(rng.uniform(0.6, 0.95)), randomness=float(rng.uniform(0.05, 0.3)),
            traj_per_cell=int(rng.choice([5, 8, 16, 33])), max_steps=int(rng.integers(300, 3000)),
            seed=(i * 104729) | (i << 40)))
        rel.append((35.0, 45.0))
    return dems, params, rel, qz


def _plain_q(dem, q, p, lo, hi):
    H, W = dem.shape
    ov = awo.Overlay(W, H, 10.0, quantised=q, levels=1)
    ov.load_dem(dem)
    ov.run(lo, hi, p)
    torch.cuda.synchronize()
    return ov.host_results()


@pytest.fixture(scope="module")
def big_batch():
    dems, params, rel, qz = _big_regions()
    b = awo.Batch(dems, 10.0, params, rel, quantised=qz)
    b.run()
    torch.cuda.synchronize()
    plain = [_plain_q(d, q, p, *r) for d, q, p, r in zip(dems, qz, params, rel)]
    return b, dems, params, rel, qz, plain


def _assert_region_equal(got, ref, stats_got, i, what=""):
    assert np.array_equal(got["count"], ref["count"]), (what, i)
    assert np.array_equal(got["maxe"], ref["maxe"]), (what, i)
    assert np.array_equal(got["vel"], ref["vel"]), (what, i)
    assert stats_got == ref["stats"], (what, i, stats_got, ref["stats"])


def test_big_regions_take_the_expected_footprint_paths(big_batch):
    b = big_batch[0]
    paths = [awo.awo_dem_gather_path(ov.h, ov.g) for ov in b.ovs]
    assert paths == [s[3] for s in BIG_SPECS]


def test_big_regions_batched_equal_plain_and_oracle(big_batch):
    b, dems, params, rel, qz, plain = big_batch
    st = b.stats_list()
    for i in range(b.n):
        got = b.results(i)
        assert np.array_equal(got["cells"], plain[i]["cells"]), i
        _assert_region_equal(got, plain[i], st[i], i, "plain")
        assert st[i]["n_traj"] > 0
    # the three regions of 2^20 cells and more, directly against the oracle
    for i in range(3):
        p = params[i]
        h = oracle.decode_u16(dems[i]) if qz[i] else dems[i]
        op = oracle.SimParams(mu=p.mu, drag_k=p.drag_k, persistence=p.persistence, randomness=p.randomness,
                              step_scale=p.step_scale, gravity=p.gravity, traj_per_cell=p.traj_per_cell,
                              max_steps=p.max_steps, seed=p.seed)
        cells = plain[i]["cells"]
        _, ref_cells = oracle.release(oracle.normals(h, 10.0, want_slope=False)[1], *rel[i])
        assert np.array_equal(cells, ref_cells), i
        c64, rm, rst = oracle.simulate_threaded(h, 10.0, cells, op)
        got = b.results(i)
        assert np.array_equal(got["count"], oracle.counts_u32(c64)), i
        assert np.array_equal(got["maxe"], rm), i
        for k in ("total_steps", "n_traj", "n_exited", "n_capped", "n_stopped"):
            assert st[i][k] == rst[k], (i, k)


def test_big_regions_every_tuning_and_graph_replay(big_batch):
    b, dems, params, rel, qz, plain = big_batch
    for rf in (awo.REFILL_LANE, awo.REFILL_WARP):
        for th in (64, 128, 256):
            for gp in (0, 256, 1024, 4096):
                b.tuning = awo.Tuning(th, gp, rf, 0)
                b.simulate()
                torch.cuda.synchronize()
                st = b.stats_list()
                for i in range(b.n):
                    ov = b.ovs[i]
                    assert np.array_equal(ov.count.cpu().numpy().view(np.uint32), plain[i]["count"]), (rf, th, gp, i)
                    assert np.array_equal(ov.maxe.cpu().numpy(), plain[i]["maxe"]), (rf, th, gp, i)
                    assert st[i] == plain[i]["stats"], (rf, th, gp, i)
    b.tuning = awo.Tuning(128, 0, awo.REFILL_LANE, 0)
    b.capture()
    for _ in range(2):
        for ov in b.ovs:
            ov.count.fill_(3)  # scribble: the replay must clear and recompute
            ov.maxe.fill_(1.0)
        b.replay()
        torch.cuda.synchronize()
        st = b.stats_list()
        for i in range(b.n):
            _assert_region_equal(b.results(i), plain[i], st[i], i, "replay")
    b.graph = None
