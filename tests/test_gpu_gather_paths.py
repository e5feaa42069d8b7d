"""The particle kernel's two ways of fetching a 2x2 footprint -- one texture
gather through a texture object over the DEM (grids of at least 2^20 cells
with a texture-aligned buffer and row pitch) and four loads (otherwise) --
give the same rasters and statistics, equal to the oracle's, including
particles that start on and run along the last row and column, where the
footprint is clamped."""
import numpy as np
import pytest
import torch

import oracle
import paper_2506_23364_gb300 as awo
from paper_2506_23364_gb300 import inputs

pytestmark = pytest.mark.gpu

H, W, CS = 1040, 1024, 10.0  # 1.06 M cells, row pitch 4096 B


def _run(dh, cells, p):
    g = awo.grid(W, H, CS)
    count = torch.zeros((H, W), dtype=torch.int32, device="cuda")
    maxe = torch.zeros((H, W), dtype=torch.float32, device="cuda")
    stats = torch.zeros(6, dtype=torch.int64, device="cuda")
    ws = torch.empty(awo.awo_simulate_workspace_bytes(cells.size), dtype=torch.uint8, device="cuda")
    dc = torch.from_numpy(cells.view(np.int32)).cuda()
    awo.awo_simulate(dh, g, dc, None, cells.size, p, count, maxe, stats, ws)
    torch.cuda.synchronize()
    return count.cpu().numpy().view(np.uint32), maxe.cpu().numpy(), awo.stats_dict(stats)


@pytest.mark.parametrize("seed", [0, 1])
def test_texture_and_load_gathers_agree_with_the_oracle(seed):
    # a DEM tilted towards the last row and column, so particles reach both borders
    z = inputs.fbm(W + 16, 0.8, seed=40 + seed, relief=900.0)[:H, :W]
    yy, xx = np.mgrid[0:H, 0:W]
    h = (z + 3000.0 - 0.9 * CS * (yy + xx)).astype(np.float32)
    rng = np.random.default_rng(seed)
    border = np.concatenate([(H - 1) * W + rng.integers(0, W, 40), rng.integers(0, H, 40) * W + (W - 1),
                             [H * W - 1, W - 1, (H - 1) * W, (H - 2) * W + W - 2]])
    cells = np.unique(np.concatenate([rng.integers(0, H * W, 300), border])).astype(np.uint32)
    op = oracle.SimParams(traj_per_cell=24, max_steps=1500, seed=(7 << 32) | seed)
    p = awo.SimParams.make(traj_per_cell=24, max_steps=1500, seed=(7 << 32) | seed)
    dh = torch.from_numpy(h).cuda()  # aligned: texture gathers
    assert dh.data_ptr() % 32 == 0
    buf = torch.zeros(H * W + 1, dtype=torch.float32, device="cuda")
    buf[1:] = dh.reshape(-1)
    dh_off = buf[1:].view(H, W)  # 4 bytes off the texture alignment: loads
    ca, ma, sa = _run(dh, cells, p)
    cb, mb, sb = _run(dh_off, cells, p)
    assert np.array_equal(ca, cb) and np.array_equal(ma, mb) and sa == sb
    c64, rm, rst = oracle.simulate_threaded(h, CS, cells, op, threads=8)
    assert np.array_equal(ca, oracle.counts_u32(c64))
    assert np.array_equal(ma, rm)
    for k in ("total_steps", "n_traj", "n_exited", "n_capped", "n_stopped"):
        assert sa[k] == rst[k], k
    # the border was reached: visits in the last row and column
    assert ca[H - 1].sum() > 0 and ca[:, W - 1].sum() > 0
    assert sa["n_exited"] > 0


def test_soft_forward_and_adjoint_same_on_both_paths():
    """Soft deposits and their adjoint: the texture-gather and the load path
    give the same fixed-point deposits and the same gradients."""
    z = inputs.fbm(W + 16, 0.8, seed=44, relief=1500.0)[:H, :W]
    h = (z + 2000.0).astype(np.float32)
    rng = np.random.default_rng(3)
    cells = np.unique(rng.integers(0, H * W, 500)).astype(np.uint32)
    n = cells.size
    p = awo.SimParams.make(traj_per_cell=16, max_steps=400, seed=11, drag_k=1e-3)
    g = awo.grid(W, H, CS)
    dc = torch.from_numpy(cells.view(np.int32)).cuda()
    wt = torch.from_numpy(rng.uniform(0.5, 1.5, n).astype(np.float32)).cuda()
    gd = torch.from_numpy(rng.normal(0, 1, (H, W)).astype(np.float32)).cuda()
    dh = torch.from_numpy(h).cuda()
    buf = torch.zeros(H * W + 1, dtype=torch.float32, device="cuda")
    buf[1:] = dh.reshape(-1)
    out = []
    for d in (dh, buf[1:].view(H, W)):
        ws = torch.empty(awo.awo_soft_workspace_bytes(n), dtype=torch.uint8, device="cuda")
        dep = torch.zeros((H, W), dtype=torch.int64, device="cuda")
        st = torch.zeros(6, dtype=torch.int64, device="cuda")
        awo.awo_soft_forward(d, g, dc, None, n, wt, p, 1.0, dep, st, ws)
        gt = torch.zeros(2, dtype=torch.float64, device="cuda")
        gw = torch.zeros(n, dtype=torch.float32, device="cuda")
        awo.awo_soft_backward(d, g, dc, None, n, wt, p, 1.0, gd, gt, gw, ws)
        torch.cuda.synchronize()
        out.append((dep.cpu().numpy(), st.cpu().numpy(), gt.cpu().numpy(), gw.cpu().numpy()))
    (da, sa, ga, wa), (db, sb, gb, wb) = out
    assert np.array_equal(da, db) and np.array_equal(sa, sb)
    # the gradients are FP64 sums of per-particle FP32 terms, added in atomic
    # order: equal up to that order's rounding
    assert np.allclose(wa, wb, rtol=1e-6, atol=0.0)
    assert np.allclose(ga, gb, rtol=1e-9, atol=0.0)
    assert int(sa[0]) > 0 and int(da.sum()) > 0


def test_first_use_of_a_buffer_inside_a_graph_capture():
    """A DEM buffer whose first particle call is being captured into a CUDA
    graph gets no new texture view (the capture must not see a call it could
    refuse): the graph runs with loads and gives the same rasters as a plain
    call, which then creates the view and gathers through it."""
    z = inputs.fbm(W + 16, 0.8, seed=45, relief=1200.0)[:H, :W]
    h = (z + 1500.0).astype(np.float32)
    rng = np.random.default_rng(9)
    cells = np.unique(rng.integers(0, H * W, 200)).astype(np.uint32)
    p = awo.SimParams.make(traj_per_cell=16, max_steps=500, seed=3, flags=1)  # clear the rasters first
    g = awo.grid(W, H, CS)
    dh = torch.from_numpy(h).cuda()  # a buffer no call has seen
    dc = torch.from_numpy(cells.view(np.int32)).cuda()
    count = torch.zeros((H, W), dtype=torch.int32, device="cuda")
    maxe = torch.zeros((H, W), dtype=torch.float32, device="cuda")
    stats = torch.zeros(6, dtype=torch.int64, device="cuda")
    ws = torch.empty(awo.awo_simulate_workspace_bytes(cells.size), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        awo.awo_simulate(dh, g, dc, None, cells.size, p, count, maxe, stats, ws)
    graph.replay()
    torch.cuda.synchronize()
    cg, mg, sg = count.cpu().numpy().view(np.uint32).copy(), maxe.cpu().numpy().copy(), awo.stats_dict(stats)
    cp, mp, sp = _run(dh, cells, p)
    assert np.array_equal(cg, cp) and np.array_equal(mg, mp) and sg == sp
    assert sg["total_steps"] > 0


def test_subnormal_heights_read_exactly():
    """Heights in the FP32 subnormal range reach the arithmetic unchanged on
    both paths (the texture view returns the DEM's words as raw bits, with
    no flush to zero), so the rasters -- energies in the subnormal range
    included -- equal the oracle's."""
    z = inputs.fbm(W + 16, 0.8, seed=46, relief=1.0)[:H, :W]
    z = (z - z.min()) / (z.max() - z.min())
    h = (z * 2.0 ** -125).astype(np.float32)  # about half below 2^-126 (subnormal)
    tiny = np.finfo(np.float32).tiny
    assert 0.1 < float(np.mean((h > 0) & (h < tiny))) < 0.9
    rng = np.random.default_rng(12)
    cells = np.unique(rng.integers(0, H * W, 400)).astype(np.uint32)
    kw = dict(traj_per_cell=8, max_steps=300, seed=13, mu=0.0)
    op = oracle.SimParams(**kw)
    p = awo.SimParams.make(**kw)
    dh = torch.from_numpy(h).cuda()
    buf = torch.zeros(H * W + 1, dtype=torch.float32, device="cuda")
    buf[1:] = dh.reshape(-1)
    ca, ma, sa = _run(dh, cells, p)
    cb, mb, sb = _run(buf[1:].view(H, W), cells, p)
    assert np.array_equal(ca, cb) and np.array_equal(ma, mb) and sa == sb
    c64, rm, rst = oracle.simulate_threaded(h, CS, cells, op, threads=8)
    assert np.array_equal(ca, oracle.counts_u32(c64))
    assert np.array_equal(ma.view(np.uint32), rm.view(np.uint32))
    assert sa["total_steps"] == rst["total_steps"] and sa["total_steps"] > 0
    assert np.any((ma > 0) & (ma < tiny))  # energies recorded in the subnormal range
