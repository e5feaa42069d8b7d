"""The largest grid the library accepts (W * H just under 2^31 cells):
normals, release, particles, velocity and mipmap on a 65536 x 32767 plane,
checked against the oracle on sampled outputs -- normals on 3 x 3 windows,
particles by their traced paths, mipmap texels on 2 x 2 windows -- plus the
release list and raster totals, which catch a wrapped 32-bit index anywhere.
About 60 GB of device memory and 8 GB of host memory."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2506_23364_gb300 as awo

pytestmark = pytest.mark.gpu

W, H, CS = 65536, 32767, 10.0
TAN_Y, TAN_X = math.tan(math.radians(35.0)), 0.05


@pytest.fixture(scope="module")
def plane():
    assert W * H < 2 ** 31
    h = np.empty((H, W), np.float32)
    x = np.arange(W, dtype=np.float64) * (CS * TAN_X)
    for y0 in range(0, H, 2048):
        y = np.arange(y0, min(y0 + 2048, H), dtype=np.float64)
        h[y0:y0 + y.size] = ((H - y)[:, None] * (CS * TAN_Y) + x[None, :]).astype(np.float32)
    dh = torch.from_numpy(h).cuda()
    yield h, dh
    del dh
    torch.cuda.empty_cache()


def test_max_grid_terrain_release(plane):
    h, dh = plane
    g = awo.grid(W, H, CS)
    t2 = torch.empty((H, W), dtype=torch.float32, device="cuda")
    awo.awo_normals(dh, g, None, t2, None)
    rng = np.random.default_rng(0)
    ys = np.concatenate([[0, H - 1, H - 1, 0, H // 2], rng.integers(0, H, 40)])
    xs = np.concatenate([[0, W - 1, 0, W - 1, W // 2], rng.integers(0, W, 40)])
    for y, x in zip(ys, xs):
        y0, y1, x0, x1 = max(y - 1, 0), min(y + 1, H - 1), max(x - 1, 0), min(x + 1, W - 1)
        _, rt, _ = oracle.normals(np.ascontiguousarray(h[y0:y1 + 1, x0:x1 + 1]), CS, want_slope=False)
        assert t2[y, x].item() == rt[y - y0, x - x0], (y, x)
    # the plane's steepness is in [30, 45] degrees everywhere: every cell is released
    n = W * H
    mask = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    cells = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(awo.awo_release_workspace_bytes(g), dtype=torch.uint8, device="cuda")
    awo.awo_release(t2, g, 30.0, 45.0, mask, cells, cnt, ws)
    torch.cuda.synchronize()
    assert int(cnt.item()) == n
    assert int(mask.sum(dtype=torch.int64).item()) == n
    idx = torch.tensor([0, 1, 2, 12345, 2 ** 30, n - 65537, n - 3, n - 2, n - 1], device="cuda")
    assert torch.equal(cells[idx].to(torch.int64), idx)
    del mask, cells, t2, ws
    torch.cuda.empty_cache()


def test_max_grid_particles_and_mipmap(plane):
    h, dh = plane
    g = awo.grid(W, H, CS)
    n = W * H
    rng = np.random.default_rng(1)
    rel = np.unique(np.concatenate([rng.integers(0, n, 200), np.arange(n - 12, n),
                                    [(H - 2) * W + W // 2, W - 1]])).astype(np.uint32)
    N, cap = 4, 300
    p = awo.SimParams.make(traj_per_cell=N, max_steps=cap, seed=(9 << 32) | 4)
    count = torch.empty((H, W), dtype=torch.int32, device="cuda")
    maxe = torch.empty((H, W), dtype=torch.float32, device="cuda")
    stats = torch.zeros(6, dtype=torch.int64, device="cuda")
    ws = torch.empty(awo.awo_simulate_workspace_bytes(rel.size), dtype=torch.uint8, device="cuda")
    p.flags = 1  # clear the rasters first
    dc = torch.from_numpy(rel.view(np.int32)).cuda()
    awo.awo_simulate(dh, g, dc, None, rel.size, p, count, maxe, stats, ws)
    # expected rasters from the oracle's traced paths
    op = oracle.SimParams(traj_per_cell=N, max_steps=cap, seed=(9 << 32) | 4)
    exp_count: dict[int, int] = {}
    exp_maxe: dict[int, float] = {}
    moves = 0
    for c in rel:
        for j in range(N):
            tr = oracle.trace(h, CS, int(c), j, op)
            moves += tr["cell"].size - 1
            for cell, e in zip(tr["cell"].tolist(), tr["e"].tolist()):
                exp_count[cell] = exp_count.get(cell, 0) + 1
                exp_maxe[cell] = max(exp_maxe.get(cell, 0.0), e)
    st = awo.stats_dict(stats)
    assert st["n_traj"] == rel.size * N and st["total_steps"] == moves
    keys = np.array(sorted(exp_count), dtype=np.int64)
    kd = torch.from_numpy(keys).cuda()
    got_c = count.view(-1)[kd].cpu().numpy().view(np.uint32)
    got_e = maxe.view(-1)[kd].cpu().numpy()
    assert np.array_equal(got_c, np.array([exp_count[k] for k in keys], np.uint32))
    assert np.array_equal(got_e, np.array([exp_maxe[k] for k in keys], np.float32))
    # nothing recorded anywhere else
    assert int(count.view(-1).to(torch.int64).sum().item()) == sum(exp_count.values())
    assert int((maxe != 0).sum().item()) == sum(1 for v in exp_maxe.values() if v != 0.0)
    # velocity and a 3-level mipmap; level 1 checked on 2 x 2 windows at the visited cells and the edges
    vel = torch.empty_like(maxe)
    awo.awo_finalize(maxe, g, 9.81, vel)
    shapes = awo.lod_shapes(g, 3)
    cl = [torch.empty(s, dtype=torch.int32, device="cuda") for s in shapes[1:]]
    vl = [torch.empty(s, dtype=torch.float32, device="cuda") for s in shapes[1:]]
    awo.awo_overlay_lod(count, vel, g, 3, cl, vl)
    torch.cuda.synchronize()
    probes = [(int(k) // W, int(k) % W) for k in keys[:: max(1, keys.size // 50)]] + [(H - 1, W - 1), (0, 0)]
    for y, x in probes:
        y0, x0 = 2 * (y // 2), 2 * (x // 2)
        wc = count[y0:y0 + 2, x0:x0 + 2].cpu().numpy().view(np.uint32)
        wv = vel[y0:y0 + 2, x0:x0 + 2].cpu().numpy()
        rc, rv = oracle.lod(wc, wv, 2)
        assert cl[0][y0 // 2, x0 // 2].item() & 0xFFFFFFFF == int(rc[1][0, 0]), (y, x)
        assert vl[0][y0 // 2, x0 // 2].item() == rv[1][0, 0], (y, x)
    assert tuple(cl[1].shape) == shapes[2]
