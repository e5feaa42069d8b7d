"""GPU parity of release evaluation on a texture of chosen resolution and of
particles started at release-texel centres (Sec. 5.2: the user picks the
texture resolution of the release evaluation), bit for bit against the
oracle, through the C ABI."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2506_23364_gb300 as awo
from paper_2506_23364_gb300 import inputs

pytestmark = pytest.mark.gpu

MU25 = math.tan(math.radians(25.0))


def _tan2(h, cs):
    """tan^2 of the DEM from the GPU's normals kernel (bit-exact to the oracle's)."""
    H, W = h.shape
    g = awo.grid(W, H, cs)
    dh = torch.from_numpy(np.ascontiguousarray(h, np.float32)).cuda()
    t2 = torch.empty((H, W), dtype=torch.float32, device="cuda")
    awo.awo_normals(dh, g, None, t2, None)
    return g, t2


def _gpu_release_texture(t2, g, r, lo, hi, mask_offset=0):
    wr, hr = awo.awo_release_texture_dims(g, r)
    raw = torch.empty(wr * hr + mask_offset, dtype=torch.uint8, device="cuda")
    mask = raw[mask_offset:]
    tex = torch.empty(wr * hr, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(awo.awo_release_texture_workspace_bytes(g, r), dtype=torch.uint8, device="cuda")
    awo.awo_release_texture(t2, g, r, lo, hi, mask, tex, n, ws)
    torch.cuda.synchronize()
    k = int(n.item())
    return mask.cpu().numpy().reshape(hr, wr), tex[:k].cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("r", [-3, -2, -1, 0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(131, 97), (1, 1), (5, 300), (64, 64)])
def test_release_texture_bitexact(r, shape):
    H, W = shape
    n = max(H, W, 8)
    h = inputs.fbm(n, 0.8, seed=H * 7 + W, relief=1500.0)[:H, :W].astype(np.float32)
    g, t2 = _tan2(h, 10.0)
    t2h = t2.cpu().numpy()
    m_ref, tex_ref = oracle.release_texture(t2h, r, 30.0, 45.0)
    m_got, tex_got = _gpu_release_texture(t2, g, r, 30.0, 45.0)
    assert np.array_equal(m_got, m_ref)
    assert np.array_equal(tex_got, tex_ref)


@pytest.mark.parametrize("r", [0, 1, 2, 3])
@pytest.mark.parametrize("W,offset", [(256, 0), (256, 1), (258, 0), (253, 0)])
def test_release_texture_load_paths(r, W, offset):
    """Runs of texels away from the row ends read the two tan^2 rows once,
    as float4 when tan2 is 16-byte aligned and W a multiple of 4 (r <= 2),
    else as scalars; the row ends take the per-texel path.  Every layout
    gives the oracle's texture."""
    H = 37
    h = inputs.fbm(W, 0.8, seed=W + r, relief=1800.0)[:H, :W].astype(np.float32)
    g, t2 = _tan2(h, 10.0)
    t2h = t2.cpu().numpy()
    buf = torch.empty(H * W + offset, dtype=torch.float32, device="cuda")
    buf[offset:] = t2.reshape(-1)
    m_ref, tex_ref = oracle.release_texture(t2h, r, 29.0, 46.0)
    m_got, tex_got = _gpu_release_texture(buf[offset:].view(H, W), g, r, 29.0, 46.0)
    assert tex_ref.size > 100
    assert np.array_equal(m_got, m_ref)
    assert np.array_equal(tex_got, tex_ref)


@pytest.mark.parametrize("r,W,H,offset", [(1, 2048, 37, 0), (1, 2048, 2, 0), (2, 1024, 19, 0), (2, 1024, 2, 1),
                                           (1, 4096, 5, 1), (2, 2048, 3, 0)])
def test_release_texture_row_groups(r, W, H, offset):
    """Textures whose rows are whole tiles (W 2^r a multiple of 4096, r = 1, 2)
    take the row-group kernel: the 2^r texture rows between two tan^2 rows
    share their horizontal interpolations, and the clamped rows at both ends
    take the per-row kernel.  Aligned and unaligned tan^2, the smallest grids
    (H = 2: one row group) and row ends included."""
    h = inputs.fbm(W, 0.8, seed=W + H + r, relief=1800.0)[:H, :W].astype(np.float32)
    g, t2 = _tan2(h, 10.0)
    t2h = t2.cpu().numpy()
    buf = torch.empty(H * W + offset, dtype=torch.float32, device="cuda")
    buf[offset:] = t2.reshape(-1)
    m_ref, tex_ref = oracle.release_texture(t2h, r, 29.0, 46.0)
    m_got, tex_got = _gpu_release_texture(buf[offset:].view(H, W), g, r, 29.0, 46.0)
    assert tex_ref.size > 100
    assert np.array_equal(m_got, m_ref)
    assert np.array_equal(tex_got, tex_ref)


def test_release_texture_unaligned_mask_and_r0():
    h = inputs.fbm(200, 0.8, seed=3, relief=1500.0).astype(np.float32)
    g, t2 = _tan2(h, 10.0)
    t2h = t2.cpu().numpy()
    m_ref, tex_ref = oracle.release_texture(t2h, 1, 28.0, 44.0)
    m_got, tex_got = _gpu_release_texture(t2, g, 1, 28.0, 44.0, mask_offset=3)
    assert np.array_equal(m_got, m_ref) and np.array_equal(tex_got, tex_ref)
    # r = 0 is the cell release
    m0, c0 = oracle.release(t2h, 28.0, 44.0)
    m_got, tex_got = _gpu_release_texture(t2, g, 0, 28.0, 44.0)
    assert np.array_equal(m_got, m0) and np.array_equal(tex_got, c0)


@pytest.mark.parametrize("r", [-2, -1, 1, 2])
def test_workflow_texels_bitexact(r):
    """decode-free workflow at a release texture of 2^r: release list,
    rasters, statistics and mipmap equal the oracle's."""
    z = inputs.fbm(160, 0.8, seed=40 + r, relief=1200.0, m=150).astype(np.float32)
    H, W = z.shape
    ov = awo.Overlay(W, H, 10.0, quantised=False, levels=3, release_log2=r)
    ov.load_dem(z)
    p = awo.SimParams.make(traj_per_cell=8, max_steps=600, seed=(5 << 32) | 9)
    ov.run(30.0, 45.0, p)
    torch.cuda.synchronize()
    got = ov.host_results()
    _, t2, _ = oracle.normals(z, 10.0)
    m_ref, tex_ref = oracle.release_texture(t2, r, 30.0, 45.0)
    op = oracle.SimParams(traj_per_cell=8, max_steps=600, seed=(5 << 32) | 9, release_log2=r)
    c64, maxe, st = oracle.simulate(z, 10.0, tex_ref, op)
    assert np.array_equal(got["mask"], m_ref)
    assert np.array_equal(got["cells"], tex_ref) and tex_ref.size > 5
    assert np.array_equal(got["count"], oracle.counts_u32(c64))
    assert np.array_equal(got["maxe"], maxe)
    for k in st:
        assert got["stats"][k] == st[k], k
    vel = oracle.finalize(maxe)
    cl, vl = oracle.lod(oracle.counts_u32(c64), vel, 3)
    for l in range(3):
        assert np.array_equal(got["count_lv"][l], cl[l]) and np.array_equal(got["vel_lv"][l], vl[l])


def test_texel_chunking_and_rejects():
    """Texel lists with few entries and many particles, and entries outside
    the texture (skipped and counted as rejected)."""
    z = inputs.fbm(96, 0.8, seed=12, relief=900.0).astype(np.float32)
    H, W = z.shape
    r = 2
    wr, hr = awo.awo_release_texture_dims(awo.grid(W, H, 10.0), r)
    rng = np.random.default_rng(2)
    tex = np.sort(rng.choice(wr * hr, 3, replace=False)).astype(np.uint32)
    bad = np.concatenate([tex, np.array([wr * hr, wr * hr + 7], np.uint32)])
    ov = awo.Overlay(W, H, 10.0, quantised=False, release_log2=r)
    ov.load_dem(z)
    dc = torch.from_numpy(bad.view(np.int32)).cuda()
    ov.simulate(awo.SimParams.make(traj_per_cell=1000, max_steps=500), cells=dc, n_cells=bad.size)
    torch.cuda.synchronize()
    c64, maxe, st = oracle.simulate(z, 10.0, tex, oracle.SimParams(traj_per_cell=1000, max_steps=500,
                                                                   release_log2=r))
    assert np.array_equal(ov.count.cpu().numpy().view(np.uint32), oracle.counts_u32(c64))
    assert np.array_equal(ov.maxe.cpu().numpy(), maxe)
    gs = ov.stats_dict()
    assert gs["n_rejected"] == 2000 and gs["n_traj"] == st["n_traj"] == 3000
    assert gs["total_steps"] == st["total_steps"]


def test_known_release_texture_from_mask():
    """A caller's release mask at the texture's resolution (known release
    points) gives the oracle's rasters for those texels."""
    z = inputs.fbm(128, 0.8, seed=8, relief=1000.0).astype(np.float32)
    H, W = z.shape
    r = 1
    ov = awo.Overlay(W, H, 10.0, quantised=False, release_log2=r)
    ov.load_dem(z)
    rng = np.random.default_rng(4)
    m = (rng.random((ov.g_rel.height, ov.g_rel.width)) < 0.01).astype(np.uint8)
    ov.terrain_from_mask(torch.from_numpy(m).cuda())
    ov.simulate(awo.SimParams.make(traj_per_cell=16, max_steps=400))
    torch.cuda.synchronize()
    tex = np.flatnonzero(m.ravel()).astype(np.uint32)
    assert np.array_equal(ov.release_cells(), tex)
    c64, maxe, _ = oracle.simulate(z, 10.0, tex, oracle.SimParams(traj_per_cell=16, max_steps=400, release_log2=r))
    assert np.array_equal(ov.count.cpu().numpy().view(np.uint32), oracle.counts_u32(c64))
    assert np.array_equal(ov.maxe.cpu().numpy(), maxe)


@pytest.mark.parametrize("refill", [awo.REFILL_LANE, awo.REFILL_WARP])
def test_batched_mixed_release_resolutions(refill):
    """One batched launch over regions whose release lists are cells (r = 0)
    and texels (r = -1, 1, 2): each region equals the oracle alone."""
    rs = [0, 1, -1, 2, 0, 1]
    dems = [inputs.fbm(64 + 32 * i, 0.8, seed=70 + i, relief=900.0).astype(np.float32) for i in range(len(rs))]
    params = [awo.SimParams.make(traj_per_cell=6 + i, max_steps=300, seed=i, release_log2=r)
              for i, r in enumerate(rs)]
    b = awo.Batch(dems, 10.0, params, [(30.0, 45.0)] * len(rs), quantised=False)
    b.tuning = awo.Tuning(128, 0, refill, 0)
    b.run()
    torch.cuda.synchronize()
    for i, (z, r) in enumerate(zip(dems, rs)):
        _, t2, _ = oracle.normals(z, 10.0)
        _, tex = oracle.release_texture(t2, r, 30.0, 45.0)
        op = oracle.SimParams(traj_per_cell=6 + i, max_steps=300, seed=i, release_log2=r)
        c64, maxe, st = oracle.simulate(z, 10.0, tex, op)
        got = b.results(i)
        assert np.array_equal(got["cells"], tex), i
        assert np.array_equal(got["count"], oracle.counts_u32(c64)), i
        assert np.array_equal(got["maxe"], maxe), i
        assert b.stats_list()[i]["total_steps"] == st["total_steps"], i


@pytest.mark.parametrize("shape,r", [((4096, 4096), 2), ((4160, 4096), 1)])
def test_release_texture_many_tiles(shape, r):
    """Textures of more than 16384 tiles of 4096 texels take the tile-count
    scan's wide path: 65536 tiles (64 a thread, 16-byte loads) and 16640
    (17 a thread, one by one)."""
    H, W = shape
    h = inputs.fbm(max(H, W), 0.8, seed=77, relief=3000.0)[:H, :W].astype(np.float32)
    g, t2 = _tan2(h, 10.0)
    wr, hr = awo.awo_release_texture_dims(g, r)
    assert (wr * hr + 4095) // 4096 > 16384
    m_ref, tex_ref = oracle.release_texture(t2.cpu().numpy(), r, 30.0, 45.0)
    m_got, tex_got = _gpu_release_texture(t2, g, r, 30.0, 45.0)
    assert np.array_equal(m_got, m_ref)
    assert np.array_equal(tex_got, tex_ref)
