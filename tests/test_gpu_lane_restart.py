"""A particle starts from its own start record whatever the particle before it
in the same lane left behind.

With randomness R = 0 a particle released on flat ground has the zero vector
as its first direction and as its move vector, so it stops at its first move
(Sec. 5.2: a zero direction ends the particle) and its lane is left with a
non-finite position.  On grids of 2^20 cells or more the footprints come by
texture gather and a lane keeps whatever position its particle ended at, so
these cases run a 1024 x 1024 staircase DEM descending along x: flat treads
two cells wide (h(x + 1) = h(x) for even x: zero first direction) and 2 m
risers at 1 m cells (odd x: the particles run down the stairs),
released from a caller mask over a block where flat and sloped cells
alternate.  Chunks of 32 particles (a quarter of a cell's at N = 128) go to warps
in any order, so lanes that ran flat-cell particles go on to sloped-cell ones.
Both the single-request and the batched kernel are compared with the oracle
bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import paper_2506_23364_gb300 as awo

pytestmark = pytest.mark.gpu

N_SIDE = 1024
CS = 1.0


def _staircase() -> np.ndarray:
    x = np.arange(N_SIDE)
    row = (2.0 * (N_SIDE // 2 - x // 2)).astype(np.float32)  # -2 m per riser, flat treads
    return np.ascontiguousarray(np.broadcast_to(row, (N_SIDE, N_SIDE)), dtype=np.float32)


def _mask() -> np.ndarray:
    m = np.zeros((N_SIDE, N_SIDE), dtype=np.uint8)
    m[400:464, 300:364] = 1  # 4096 cells, even x flat, odd x sloped
    return m


def _params(**kw):
    base = dict(randomness=0.0, persistence=0.9, traj_per_cell=128, max_steps=64, seed=11)
    base.update(kw)
    return base


def _oracle(dem, mask, kw):
    cells = np.flatnonzero(mask.ravel()).astype(np.uint32)
    op = oracle.SimParams(**kw)
    count64, maxe, st = oracle.simulate_threaded(dem, CS, cells, op)
    return oracle.counts_u32(count64), maxe, st


def test_flat_release_cells_have_zero_first_direction():
    """The case is the one described: flat-cell particles stop at their first move."""
    dem = _staircase()
    st_flat = oracle.trace(dem, CS, 420 * N_SIDE + 310, 0, oracle.SimParams(**_params()))
    st_slope = oracle.trace(dem, CS, 420 * N_SIDE + 311, 0, oracle.SimParams(**_params()))
    assert st_flat["u"].size == 1 and st_flat["end"] == "stopped"
    assert st_slope["u"].size > 1


@pytest.mark.parametrize("kw", [_params(), _params(persistence=0.0, seed=3), _params(traj_per_cell=33, seed=5)])
def test_single_request_restart_after_zero_direction(kw):
    dem, mask = _staircase(), _mask()
    ov = awo.Overlay(N_SIDE, N_SIDE, CS, quantised=False, levels=1, want_normals=False, want_mask=False)
    ov.load_dem(dem)
    assert awo.awo_dem_gather_path(ov.h, ov.g) == "texture"
    ov.terrain_from_mask(torch.from_numpy(mask).cuda())
    ov.simulate(awo.SimParams.make(**kw))
    torch.cuda.synchronize()
    count, maxe, st = _oracle(dem, mask, kw)
    got = ov.stats_dict()
    assert {k: got[k] for k in st} == st
    assert np.array_equal(ov.count.cpu().numpy().view(np.uint32), count)
    assert np.array_equal(ov.maxe.cpu().numpy(), maxe)


def test_batched_restart_after_zero_direction():
    dem, mask = _staircase(), _mask()
    kws = [_params(), _params(persistence=0.5, traj_per_cell=64, seed=9)]
    b = awo.Batch([dem, dem], CS, [awo.SimParams.make(**kw) for kw in kws], [(0.0, 90.0)] * 2, quantised=False)
    for ov in b.ovs:
        ov.terrain_from_mask(torch.from_numpy(mask).cuda())
    b.simulate()
    torch.cuda.synchronize()
    st_all = b.stats_list()
    for i, kw in enumerate(kws):
        count, maxe, st = _oracle(dem, mask, kw)
        assert {k: st_all[i][k] for k in st} == st, i
        assert np.array_equal(b.ovs[i].count.cpu().numpy().view(np.uint32), count), i
        assert np.array_equal(b.ovs[i].maxe.cpu().numpy(), maxe), i
