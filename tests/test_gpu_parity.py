"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Counts, release lists, masks and every FP32 raster are compared bit for bit:
the kernels and the oracle evaluate the same IEEE-754 FP32 operations in the
same order with no fused multiply-add.  Only slope_deg (atanf, display only)
has a tolerance.  Inputs are the seeded synthetic workloads (tiny, mid, the
large DEM's 1024^2 crop, and the full 8192^2 DEM with sampled release cells).
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2506_23364_gb300 as awo
from paper_2506_23364_gb300 import inputs

pytestmark = pytest.mark.gpu

MU25 = math.tan(math.radians(25.0))


def _oparams(w=None, **kw):
    base = dict(mu=MU25, drag_k=0.0, persistence=0.9, randomness=0.16, step_scale=1.0, gravity=9.81,
                traj_per_cell=16, max_steps=1000, seed=0)
    if w is not None:
        base.update(mu=w.mu, drag_k=w.drag_k, persistence=w.persistence, randomness=w.randomness,
                    step_scale=w.step_scale, gravity=w.gravity, traj_per_cell=w.traj_per_cell,
                    max_steps=w.max_steps, seed=w.seed)
    base.update(kw)
    return oracle.SimParams(**base)


def _gparams(op: oracle.SimParams) -> awo.SimParams:
    return awo.SimParams.make(mu=op.mu, drag_k=op.drag_k, persistence=op.persistence, randomness=op.randomness,
                              step_scale=op.step_scale, gravity=op.gravity, traj_per_cell=op.traj_per_cell,
                              max_steps=op.max_steps, seed=op.seed)


def _oracle_workflow(dem, cs, quantised, lo, hi, op, levels, cells=None):
    h = oracle.decode_u16(dem, inputs.DECODE_SCALE) if quantised else np.asarray(dem, np.float32)
    nrm, t2, sd = oracle.normals(h, cs)
    mask, rel = oracle.release(t2, lo, hi)
    sim_cells = rel if cells is None else cells
    c64, maxe, st = oracle.simulate_threaded(h, cs, sim_cells, op)
    count = oracle.counts_u32(c64)
    vel = oracle.finalize(maxe, op.gravity)
    cl, vl = oracle.lod(count, vel, levels)
    return {"h": h, "normals": nrm, "tan2": t2, "slope_deg": sd, "mask": mask, "cells": rel, "count": count,
            "maxe": maxe, "vel": vel, "count_lv": cl, "vel_lv": vl, "stats": st}


def _gpu_workflow(dem, cs, quantised, lo, hi, op, levels, cells=None):
    H, W = dem.shape
    ov = awo.Overlay(W, H, cs, quantised=quantised, levels=levels, want_slope=True)
    ov.load_dem(dem)
    p = _gparams(op)
    ov.terrain(lo, hi, inputs.DECODE_SCALE)
    if cells is None:
        ov.simulate(p)
    else:
        dc = torch.from_numpy(np.ascontiguousarray(cells, np.uint32).view(np.int32)).cuda()
        ov.simulate(p, cells=dc, n_cells=cells.size)
    ov.overlay(op.gravity)
    torch.cuda.synchronize()
    return ov.host_results()


def _assert_same(got, ref, what=("cells", "mask", "tan2", "normals", "count", "maxe", "vel")):
    for k in what:
        a, b = got[k], ref[k]
        assert a.shape == b.shape, (k, a.shape, b.shape)
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            raise AssertionError(f"{k}: {bad.shape[0]} elements differ, first at {bad[0].tolist()}: "
                                 f"gpu {a[tuple(bad[0])]!r} oracle {b[tuple(bad[0])]!r}")
    assert np.allclose(got["slope_deg"], ref["slope_deg"], rtol=1e-6, atol=1e-5)
    for l in range(len(ref["count_lv"])):
        assert np.array_equal(got["count_lv"][l], ref["count_lv"][l]), f"count level {l}"
        assert np.array_equal(got["vel_lv"][l], ref["vel_lv"][l]), f"vel level {l}"
    gs, rs = got["stats"], ref["stats"]
    for k in ("total_steps", "n_traj", "n_exited", "n_capped", "n_stopped"):
        assert gs[k] == rs[k], (k, gs[k], rs[k])
    assert gs["n_rejected"] == 0
    assert int(got["count"].astype(np.uint64).sum()) == gs["n_traj"] + gs["total_steps"]


@pytest.fixture(scope="session")
def large_dem():
    return inputs.large_dem_u16()


# ----------------------------------------------------------------------------
# Stages
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(1000, 777), (1, 1), (3, 4099)])
def test_decode_bitexact(shape):
    rng = np.random.default_rng(1)
    q = rng.integers(0, 65536, size=shape, dtype=np.uint16)
    H, W = shape
    g = awo.grid(W, H, 10.0)
    dq = torch.from_numpy(q.view(np.int16)).cuda()
    dh = torch.empty(shape, dtype=torch.float32, device="cuda")
    awo.awo_decode_u16(dq, g, 0.1, dh)
    assert np.array_equal(dh.cpu().numpy(), oracle.decode_u16(q, 0.1))


@pytest.mark.parametrize("shape", [(256, 256), (257, 300), (1, 1), (1, 37), (41, 1), (5, 3), (1024, 1031)])
def test_normals_bitexact(shape):
    H, W = shape
    rng = np.random.default_rng(H * 7 + W)
    h = (inputs.fbm(max(H, 2), 0.8, seed=H + W, relief=800.0, m=max(W, 2))[:H, :W]
         + rng.normal(0, 0.5, size=(H, W))).astype(np.float32)
    g = awo.grid(W, H, 7.5)
    dh = torch.from_numpy(h).cuda()
    nrm = torch.empty((3, H, W), dtype=torch.float32, device="cuda")
    t2 = torch.empty((H, W), dtype=torch.float32, device="cuda")
    sd = torch.empty((H, W), dtype=torch.float32, device="cuda")
    awo.awo_normals(dh, g, nrm, t2, sd)
    rn, rt, rs = oracle.normals(h, 7.5)
    assert np.array_equal(nrm.cpu().numpy(), rn)
    assert np.array_equal(t2.cpu().numpy(), rt)
    assert np.allclose(sd.cpu().numpy(), rs, rtol=1e-6, atol=1e-5)


@pytest.mark.parametrize("shape,lo,hi", [((256, 256), 30.0, 45.0), ((257, 300), 10.0, 20.0), ((1, 1), 0.0, 89.0),
                                         ((77, 53), 80.0, 85.0), ((64, 64), 0.0, 89.9), ((1, 4097), 5.0, 50.0),
                                         ((2048, 2049), 35.0, 40.0)])
def test_release_bitexact(shape, lo, hi):
    H, W = shape
    rng = np.random.default_rng(H + 3 * W)
    t2 = (rng.uniform(0, 1.3, size=(H, W)) ** 2).astype(np.float32)
    g = awo.grid(W, H, 10.0)
    dt = torch.from_numpy(t2).cuda()
    mask = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    cells = torch.empty(H * W, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(awo.awo_release_workspace_bytes(g), dtype=torch.uint8, device="cuda")
    awo.awo_release(dt, g, lo, hi, mask, cells, n, ws)
    rm, rc = oracle.release(t2, lo, hi)
    k = int(n.item())
    assert k == rc.size
    assert np.array_equal(mask.cpu().numpy(), rm)
    assert np.array_equal(cells[:k].cpu().numpy().view(np.uint32), rc)


def test_release_unaligned_mask():
    H, W = 33, 129
    rng = np.random.default_rng(5)
    t2 = (rng.uniform(0, 1.3, size=(H, W)) ** 2).astype(np.float32)
    g = awo.grid(W, H, 10.0)
    buf = torch.zeros(H * W + 17, dtype=torch.uint8, device="cuda")
    mask = buf[3:3 + H * W]
    cells = torch.empty(H * W, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(awo.awo_release_workspace_bytes(g), dtype=torch.uint8, device="cuda")
    awo.awo_release(torch.from_numpy(t2).cuda(), g, 20.0, 40.0, mask, cells, n, ws)
    rm, rc = oracle.release(t2, 20.0, 40.0)
    assert np.array_equal(mask.cpu().numpy().reshape(H, W), rm)
    assert np.array_equal(buf[:3].cpu().numpy(), np.zeros(3, np.uint8))
    assert np.array_equal(buf[3 + H * W:].cpu().numpy(), np.zeros(14, np.uint8))
    assert np.array_equal(cells[:int(n.item())].cpu().numpy().view(np.uint32), rc)


@pytest.mark.parametrize("shape,levels", [((300, 257), 9), ((1, 1), 3), ((64, 64), 7), ((1000, 3), 16)])
def test_finalize_and_lod_bitexact(shape, levels):
    H, W = shape
    rng = np.random.default_rng(W)
    cnt = rng.integers(0, 1000, size=(H, W), dtype=np.uint64).astype(np.uint32)
    big = rng.random((H, W)) < 0.2  # some blocks saturate at 2^32-1
    cnt[big] = rng.integers(2 ** 30, 2 ** 32, size=int(big.sum()), dtype=np.uint64).astype(np.uint32)
    maxe = rng.uniform(0, 300, size=(H, W)).astype(np.float32)
    maxe[rng.random((H, W)) < 0.3] = 0
    g = awo.grid(W, H, 10.0)
    dm = torch.from_numpy(maxe).cuda()
    dv = torch.empty_like(dm)
    awo.awo_finalize(dm, g, 9.81, dv)
    vel = oracle.finalize(maxe, 9.81)
    assert np.array_equal(dv.cpu().numpy(), vel)
    shapes = awo.lod_shapes(g, levels)
    cl = [torch.empty(s, dtype=torch.int32, device="cuda") for s in shapes[1:]]
    vl = [torch.empty(s, dtype=torch.float32, device="cuda") for s in shapes[1:]]
    dc = torch.from_numpy(cnt.view(np.int32)).cuda()
    awo.awo_overlay_lod(dc, dv, g, levels, cl, vl)
    rc, rv = oracle.lod(cnt, vel, levels)
    for l in range(1, levels):
        assert np.array_equal(cl[l - 1].cpu().numpy().view(np.uint32), rc[l]), l
        assert np.array_equal(vl[l - 1].cpu().numpy(), rv[l]), l


# ----------------------------------------------------------------------------
# Whole workflow
# ----------------------------------------------------------------------------
def test_tiny_workflow_bitexact():
    w = inputs.tiny()
    op = _oparams(w)
    got = _gpu_workflow(w.dem_f32, w.cell_size, False, w.slope_lo_deg, w.slope_hi_deg, op, 4)
    ref = _oracle_workflow(w.dem_f32, w.cell_size, False, w.slope_lo_deg, w.slope_hi_deg, op, 4)
    _assert_same(got, ref)
    assert got["stats"]["n_traj"] == 16 * ref["cells"].size > 10 ** 6


def test_mid_workflow_bitexact():
    w = inputs.mid()
    op = _oparams(w)
    got = _gpu_workflow(w.dem_u16, w.cell_size, True, w.slope_lo_deg, w.slope_hi_deg, op, 5)
    ref = _oracle_workflow(w.dem_u16, w.cell_size, True, w.slope_lo_deg, w.slope_hi_deg, op, 5)
    assert np.array_equal(got["h"], ref["h"])
    _assert_same(got, ref)
    assert 0.04 < ref["cells"].size / ref["h"].size < 0.06


def test_large_crop_workflow_bitexact(large_dem):
    w = inputs.crop(inputs.Workload("large", 8192, 8192, inputs.CELL_SIZE_M, *inputs.LARGE_RELEASE_DEG,
                                    traj_per_cell=256, max_steps=8000, lod_levels=6, dem_u16=large_dem), 1024)
    op = _oparams(w)
    got = _gpu_workflow(w.dem_u16, w.cell_size, True, w.slope_lo_deg, w.slope_hi_deg, op, 6)
    ref = _oracle_workflow(w.dem_u16, w.cell_size, True, w.slope_lo_deg, w.slope_hi_deg, op, 6)
    _assert_same(got, ref)


def test_large_full_size_sampled(large_dem):
    """8192^2 in the benchmark's launch configuration: terrain stages bit-exact
    over the whole grid; the full particle run (3.36 M release cells x 256
    particles) checked by its invariants and then cell by cell against the
    oracle's rasters and statistics (the oracle on every host core, about 15 s
    on 16); and a sample of 3000 release cells run alone, bit-exact."""
    n = 8192
    lo, hi = inputs.LARGE_RELEASE_DEG
    op = _oparams(traj_per_cell=256, max_steps=8000)
    ov = awo.Overlay(n, n, inputs.CELL_SIZE_M, quantised=True, levels=6)
    ov.load_dem(large_dem)
    ov.run(lo, hi, _gparams(op))
    torch.cuda.synchronize()
    st = ov.stats_dict()
    h = oracle.decode_u16(large_dem)
    assert np.array_equal(ov.h.cpu().numpy(), h)
    _, t2, _ = oracle.normals(h, inputs.CELL_SIZE_M, want_slope=False)
    assert np.array_equal(ov.tan2.cpu().numpy(), t2)
    mask, rel = oracle.release(t2, lo, hi)
    assert np.array_equal(ov.mask.cpu().numpy(), mask)
    assert np.array_equal(ov.release_cells(), rel)
    cnt = ov.count.cpu().numpy().view(np.uint32)
    assert st["n_traj"] == 256 * rel.size and st["n_rejected"] == 0
    assert int(cnt.astype(np.uint64).sum()) == st["n_traj"] + st["total_steps"]
    assert st["n_traj"] == st["n_exited"] + st["n_capped"] + st["n_stopped"]
    maxe = ov.maxe.cpu().numpy()
    assert np.all(maxe >= 0) and np.all(maxe[cnt == 0] == 0)
    vel = ov.vel.cpu().numpy()
    assert np.array_equal(vel, oracle.finalize(maxe))
    cl, vl = oracle.lod(cnt, vel, 6)
    for l in range(1, 6):
        assert np.array_equal(ov.count_lv[l - 1].cpu().numpy().view(np.uint32), cl[l])
        assert np.array_equal(ov.vel_lv[l - 1].cpu().numpy(), vl[l])
    # every cell of the full run against the oracle
    threads = min(16, os.cpu_count() or 1)
    c64_all, maxe_all, st_all = oracle.simulate_threaded(h, inputs.CELL_SIZE_M, rel, op, threads=threads)
    assert np.array_equal(cnt, oracle.counts_u32(c64_all))
    del c64_all
    assert np.array_equal(maxe, maxe_all)
    del maxe_all
    for k in ("total_steps", "n_traj", "n_exited", "n_capped", "n_stopped"):
        assert st[k] == st_all[k], k
    # sampled release cells, same kernel and launch shape
    rng = np.random.default_rng(0)
    sub = np.sort(rng.choice(rel, 3000, replace=False)).astype(np.uint32)
    dc = torch.from_numpy(sub.view(np.int32)).cuda()
    ov.simulate(_gparams(op), cells=dc, n_cells=sub.size)
    torch.cuda.synchronize()
    c64, rmaxe, rst = oracle.simulate_threaded(h, inputs.CELL_SIZE_M, sub, op, threads=4)
    assert np.array_equal(ov.count.cpu().numpy().view(np.uint32), oracle.counts_u32(c64))
    assert np.array_equal(ov.maxe.cpu().numpy(), rmaxe)
    assert ov.stats_dict()["total_steps"] == rst["total_steps"]


# ----------------------------------------------------------------------------
# Edge cases of the particle kernel
# ----------------------------------------------------------------------------
def _sim_pair(h, cs, cells, op, clear=True, ov=None):
    H, W = h.shape
    if ov is None:
        ov = awo.Overlay(W, H, cs, quantised=False)
        ov.load_dem(h)
    dc = torch.from_numpy(np.ascontiguousarray(cells, np.uint32).view(np.int32)).cuda() if cells.size else \
        torch.zeros(1, dtype=torch.int32, device="cuda")
    ov.simulate(_gparams(op), clear=clear, cells=dc, n_cells=cells.size)
    torch.cuda.synchronize()
    return ov


@pytest.mark.parametrize("kw", [dict(max_steps=0), dict(traj_per_cell=0), dict(step_scale=0.5),
                                dict(drag_k=1e-3), dict(randomness=0.0, persistence=1.0),
                                dict(randomness=0.0, persistence=0.0), dict(seed=(123 << 32) | 77),
                                dict(randomness=1.5, persistence=0.3), dict(traj_per_cell=33, max_steps=17),
                                dict(mu=0.0, max_steps=50)])
def test_simulate_parameter_cases(kw):
    z = inputs.fbm(96, 0.8, seed=9, relief=900.0, m=131).astype(np.float32)
    H, W = z.shape
    rng = np.random.default_rng(1)
    cells = np.sort(rng.choice(W * H, 400, replace=False)).astype(np.uint32)
    op = _oparams(**kw)
    ov = _sim_pair(z, 10.0, cells, op)
    c64, maxe, st = oracle.simulate(z, 10.0, cells, op)
    assert np.array_equal(ov.count.cpu().numpy().view(np.uint32), oracle.counts_u32(c64))
    assert np.array_equal(ov.maxe.cpu().numpy(), maxe)
    gs = ov.stats_dict()
    for k in st:
        assert gs[k] == st[k], k


@pytest.mark.parametrize("n_cells,N", [(1, 1000), (3, 2048), (2, 37), (5000, 1), (700, 3)])
def test_simulate_chunking(n_cells, N):
    """Work is handed out in chunks of particles that may split a release
    cell or span many: a few cells with many particles, and many cells with
    one or three particles, give the oracle's rasters bit for bit."""
    z = inputs.fbm(96, 0.8, seed=21, relief=900.0, m=131).astype(np.float32)
    H, W = z.shape
    rng = np.random.default_rng(n_cells * 7 + N)
    cells = np.sort(rng.choice(W * H, n_cells, replace=False)).astype(np.uint32)
    op = _oparams(traj_per_cell=N, max_steps=400)
    ov = _sim_pair(z, 10.0, cells, op)
    c64, maxe, st = oracle.simulate(z, 10.0, cells, op)
    assert np.array_equal(ov.count.cpu().numpy().view(np.uint32), oracle.counts_u32(c64))
    assert np.array_equal(ov.maxe.cpu().numpy(), maxe)
    gs = ov.stats_dict()
    for k in st:
        assert gs[k] == st[k], k


@pytest.mark.parametrize("shape", [(1, 1), (2, 2), (1, 40), (40, 1), (3, 5)])
def test_simulate_tiny_grids(shape):
    H, W = shape
    rng = np.random.default_rng(W * 10 + H)
    z = (1000.0 - 8.0 * np.arange(H)[:, None] - 3.0 * np.arange(W)[None, :]
         + rng.normal(0, 1.0, size=(H, W))).astype(np.float32)
    cells = np.arange(W * H, dtype=np.uint32)
    op = _oparams(traj_per_cell=8, max_steps=100)
    ov = _sim_pair(z, 5.0, cells, op)
    c64, maxe, st = oracle.simulate(z, 5.0, cells, op)
    assert np.array_equal(ov.count.cpu().numpy().view(np.uint32), oracle.counts_u32(c64))
    assert np.array_equal(ov.maxe.cpu().numpy(), maxe)
    assert ov.stats_dict()["total_steps"] == st["total_steps"]


def test_simulate_empty_list_and_device_count():
    z = inputs.plane(50, 60, 10.0, math.tan(math.radians(35.0))).astype(np.float32)
    op = _oparams()
    ov = _sim_pair(z, 10.0, np.zeros(0, np.uint32), op)
    assert ov.stats_dict()["n_traj"] == 0 and int(ov.count.sum().item()) == 0
    # device-side count smaller than the host maximum
    cells = np.arange(0, 50 * 59, 13, dtype=np.uint32)
    dc = torch.from_numpy(cells.view(np.int32)).cuda()
    ndev = torch.tensor([37], dtype=torch.int32, device="cuda")
    p = _gparams(op)
    p.flags = 1
    awo.awo_simulate(ov.h, ov.g, dc, ndev, cells.size, p, ov.count, ov.maxe, ov.stats, ov.ws_sim)
    torch.cuda.synchronize()
    c64, maxe, st = oracle.simulate(z, 10.0, cells[:37], op)
    assert np.array_equal(ov.count.cpu().numpy().view(np.uint32), oracle.counts_u32(c64))
    assert ov.stats_dict()["n_traj"] == 37 * op.traj_per_cell


def test_simulate_accumulates_and_rejects_bad_cells():
    z = inputs.fbm(64, 0.8, seed=4, relief=700.0).astype(np.float32)
    op = _oparams(traj_per_cell=4, max_steps=300)
    a = np.arange(0, 64 * 64, 11, dtype=np.uint32)
    b = np.arange(5, 64 * 64, 17, dtype=np.uint32)
    ov = _sim_pair(z, 10.0, a, op)
    ov = _sim_pair(z, 10.0, b, op, clear=False, ov=ov)
    c64, maxe, _ = oracle.simulate(z, 10.0, a, op)
    c64, maxe, _ = oracle.simulate(z, 10.0, b, op, count64=c64, maxe=maxe)
    assert np.array_equal(ov.count.cpu().numpy().view(np.uint32), oracle.counts_u32(c64))
    assert np.array_equal(ov.maxe.cpu().numpy(), maxe)
    bad = np.array([3, 64 * 64, 10, 2 ** 31 + 5], dtype=np.uint32)
    ov = _sim_pair(z, 10.0, bad, op)
    st = ov.stats_dict()
    assert st["n_rejected"] == 2 * op.traj_per_cell and st["n_traj"] == 2 * op.traj_per_cell
    c64, _, _ = oracle.simulate(z, 10.0, bad[[0, 2]], op)
    assert np.array_equal(ov.count.cpu().numpy().view(np.uint32), oracle.counts_u32(c64))


def test_side_stream_and_determinism():
    w = inputs.tiny()
    op = _oparams(w, traj_per_cell=4)
    s = torch.cuda.Stream()
    outs = []
    for _ in range(2):
        ov = awo.Overlay(256, 256, 10.0, quantised=False, levels=3)
        with torch.cuda.stream(s):
            ov.load_dem(w.dem_f32)
            ov.run(30.0, 45.0, _gparams(op))
        s.synchronize()
        outs.append(ov.host_results())
    for k in ("count", "maxe", "vel", "cells"):
        assert np.array_equal(outs[0][k], outs[1][k])


def test_gpu_errors_are_statuses():
    g = awo.grid(16, 16, 10.0)
    h = torch.zeros((16, 16), dtype=torch.float32, device="cuda")
    cnt = torch.zeros((16, 16), dtype=torch.int32, device="cuda")
    ws = torch.empty(8, dtype=torch.uint8, device="cuda")
    cells = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(awo.AwoError) as ei:
        awo.awo_simulate(h, g, cells, None, 4, awo.SimParams.make(), cnt, h, None, ws)
    assert ei.value.status == awo.AWO_ENOMEM
    ws = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(awo.AwoError) as ei:
        awo.awo_simulate(h, g, cells, None, 4, awo.SimParams.make(persistence=2.0), cnt, h, None, ws)
    assert ei.value.status == awo.AWO_EINVAL
