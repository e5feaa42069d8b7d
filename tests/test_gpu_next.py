"""GPU parity of the next-row features: release from a caller's mask, the
parabola-shaped stand-in workflow, compose colouring / blending and the
snow-cover mask (all bit for bit against the oracle)."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2506_23364_gb300 as awo
from paper_2506_23364_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,density", [((257, 300), 0.05), ((1, 1), 1.0), ((33, 129), 0.0), ((64, 64), 1.0),
                                           ((1000, 999), 0.3)])
def test_release_from_mask(shape, density):
    H, W = shape
    rng = np.random.default_rng(H + W)
    m = (rng.random((H, W)) < density).astype(np.uint8) * rng.integers(1, 256, (H, W)).astype(np.uint8)
    g = awo.grid(W, H, 10.0)
    cells = torch.empty(H * W, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(awo.awo_release_workspace_bytes(g), dtype=torch.uint8, device="cuda")
    awo.awo_release_from_mask(torch.from_numpy(m).cuda(), g, cells, n, ws)
    k = int(n.item())
    want = np.flatnonzero(m.ravel())
    assert k == want.size
    assert np.array_equal(cells[:k].cpu().numpy().view(np.uint32), want.astype(np.uint32))


def test_parabola_standin_bitexact():
    w = inputs.parabola()
    mask = inputs.parabola_release_mask()
    ov = awo.Overlay(w.width, w.height, w.cell_size, quantised=False, levels=3)
    ov.load_dem(w.dem_f32)
    p = awo.SimParams.make(traj_per_cell=w.traj_per_cell, max_steps=w.max_steps, seed=w.seed)
    ov.terrain_from_mask(torch.from_numpy(mask).cuda())
    ov.simulate(p)
    ov.overlay(w.gravity)
    torch.cuda.synchronize()
    got = ov.host_results()
    cells = np.flatnonzero(mask.ravel()).astype(np.uint32)
    c64, maxe, st = oracle.simulate_threaded(w.dem_f32, w.cell_size, cells,
                                             oracle.SimParams(traj_per_cell=w.traj_per_cell, max_steps=w.max_steps))
    assert np.array_equal(got["cells"], cells)
    assert np.array_equal(got["count"], oracle.counts_u32(c64))
    assert np.array_equal(got["maxe"], maxe)
    assert got["stats"]["n_traj"] == 6144 and got["stats"]["total_steps"] == st["total_steps"]


RAMPS = {
    "velocity5": awo.VELOCITY_STOPS,
    "two": [(0.0, (0, 0, 0)), (1.0, (255, 128, 1))],
    "ramp16": [(float(3 * i * i), (16 * i, 255 - 16 * i, (37 * i) % 256)) for i in range(16)],
    "huge": [(-1.0e30, (10, 20, 30)), (0.0, (200, 0, 100)), (1.0e30, (0, 255, 0))],  # widths above 2^60
    "tiny": [(0.0, (0, 0, 255)), (1.0e-20, (255, 0, 0)), (2.5e-20, (0, 255, 0)), (6.0e-20, (9, 9, 9))],
}


@pytest.mark.parametrize("ramp", sorted(RAMPS))
@pytest.mark.parametrize("with_base", [False, True])
def test_compose_bitexact(ramp, with_base):
    """Every stop count has its own kernel instance and the division of the
    ramp has a fast path for widths in [2^-60, 2^60]: stop counts 2..16,
    widths inside and outside that range, values on the stops, between them
    and beyond both ends."""
    stops = RAMPS[ramp]
    rng = np.random.default_rng(5)
    H, W = 301, 257
    lo, hi = stops[0][0], stops[-1][0]
    pad = 0.1 * (hi - lo)
    v = rng.uniform(lo - pad, hi + pad, (H, W)).astype(np.float32)
    on = rng.random((H, W)) < 0.05
    v[on] = np.array([s[0] for s in stops], dtype=np.float32)[rng.integers(0, len(stops), int(on.sum()))]
    v[rng.random((H, W)) < 0.02] = np.float32(lo)
    cnt = rng.integers(0, 5, (H, W)).astype(np.uint32)
    base = rng.integers(0, 256, (H, W, 4)).astype(np.uint8) if with_base else None
    g = awo.grid(W, H, 10.0)
    cm = awo.Colormap.make(stops, alpha=0.7, count_min=2)
    out = torch.empty((H, W, 4), dtype=torch.uint8, device="cuda")
    awo.awo_compose(torch.from_numpy(v).cuda(), torch.from_numpy(cnt.view(np.int32)).cuda(), g, cm,
                    torch.from_numpy(base).cuda() if with_base else None, out)
    want = oracle.compose(v, cnt, stops, 0.7, 2, base)
    assert np.array_equal(out.cpu().numpy(), want)


def test_compose_unaligned_buffers():
    """Buffers off the 16-byte boundary take the one-texel path."""
    rng = np.random.default_rng(8)
    H, W = 37, 53
    v = rng.uniform(-5, 80, (H * W + 1,)).astype(np.float32)
    cnt = rng.integers(0, 5, (H * W + 1,)).astype(np.uint32)
    base = rng.integers(0, 256, (H * W + 1, 4)).astype(np.uint8)
    dv, dc, db = torch.from_numpy(v).cuda(), torch.from_numpy(cnt.view(np.int32)).cuda(), torch.from_numpy(base).cuda()
    out = torch.empty((H * W + 1, 4), dtype=torch.uint8, device="cuda")
    cm = awo.Colormap.make(awo.VELOCITY_STOPS, alpha=0.7, count_min=2)
    awo.awo_compose(dv[1:], dc[1:], awo.grid(W, H, 10.0), cm, db[1:], out[1:])
    want = oracle.compose(v[1:].reshape(H, W), cnt[1:].reshape(H, W), awo.VELOCITY_STOPS, 0.7, 2,
                          base[1:].reshape(H, W, 4))
    assert np.array_equal(out[1:].cpu().numpy().reshape(H, W, 4), want)


def test_snow_cover_bitexact():
    w = inputs.tiny()
    h = w.dem_f32
    H, W = h.shape
    g = awo.grid(W, H, w.cell_size)
    dh = torch.from_numpy(h).cuda()
    nrm = torch.empty((3, H, W), dtype=torch.float32, device="cuda")
    awo.awo_normals(dh, g, nrm, None, None)
    p = awo.SnowParams(1500.0, 300.0, 36.0, 4.0)
    a = torch.empty((H, W), dtype=torch.float32, device="cuda")
    rgba = torch.empty((H, W, 4), dtype=torch.uint8, device="cuda")
    awo.awo_snow_cover(dh, nrm[2].contiguous(), g, p, a, rgba)
    rn, _, _ = oracle.normals(h, w.cell_size)
    ra, rrgba = oracle.snow_cover(h, rn[2], 1500.0, 300.0, 36.0, 4.0)
    assert np.array_equal(a.cpu().numpy(), ra)
    assert np.array_equal(rgba.cpu().numpy(), rrgba)
    assert 0.0 < ra.mean() < 1.0


def test_overlay_graph_replay_bitexact():
    """The whole single-region workflow captured in a CUDA graph and replayed
    on a second DEM gives the oracle's overlay for that DEM."""
    w = inputs.mid()
    dem2 = inputs.fbm(512, 0.8, seed=77, relief=1500.0)
    q2 = inputs.quantise_dm(dem2)
    cw = inputs.crop(w, 512)
    ov = awo.Overlay(512, 512, cw.cell_size, quantised=True, levels=3)
    ov.load_dem(cw.dem_u16)
    p = awo.SimParams.make(traj_per_cell=8, max_steps=500, seed=3)
    ov.capture(30.0, 45.0, p)
    ov.load_dem(q2)
    ov.replay()
    torch.cuda.synchronize()
    got = ov.host_results()
    h = oracle.decode_u16(q2)
    ref = oracle.overlay(h, cw.cell_size, 30.0, 45.0, oracle.SimParams(traj_per_cell=8, max_steps=500, seed=3), 3)
    assert np.array_equal(got["cells"], ref["cells"])
    assert np.array_equal(got["count"], ref["count"]) and np.array_equal(got["vel"], ref["vel"])
    for l in range(3):
        assert np.array_equal(got["count_lv"][l], ref["count_lv"][l])
        assert np.array_equal(got["vel_lv"][l], ref["vel_lv"][l])
