"""Invariants of the trajectory model, checked on the FP32 oracle.

(i) the count raster sums to trajectories + recorded moves; (ii) with no drag
every visit lies below the release point's energy line, so nothing is recorded
upslope of release; (iii) a move that climbs never gains energy; (iv) velocity
is bounded by sqrt(2 g relief).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2506_23364_gb300 import inputs
from tests import fp64_paths

MU25 = math.tan(math.radians(25.0))


@pytest.fixture(scope="module")
def fbm_small():
    z = inputs.fbm(96, 0.8, seed=5, relief=600.0, m=80)
    q = inputs.quantise_dm(z)
    h = oracle.decode_u16(q)
    _, t2, _ = oracle.normals(h, 10.0)
    _, cells = oracle.release(t2, 30.0, 45.0)
    return h, cells


def test_count_conservation_and_velocity_bound(fbm_small):
    h, cells = fbm_small
    p = oracle.SimParams(mu=MU25, traj_per_cell=8, max_steps=500, seed=3)
    c64, maxe, st = oracle.simulate(h, 10.0, cells, p)
    assert cells.size > 100
    assert c64.sum() == st["n_traj"] + st["total_steps"]
    assert st["n_traj"] == 8 * cells.size
    assert st["n_traj"] == st["n_exited"] + st["n_capped"] + st["n_stopped"]
    vel = oracle.finalize(maxe)
    relief = float(h.max() - h.min())
    assert vel.max() <= math.sqrt(2 * 9.81 * relief)
    assert np.all(maxe[c64 == 0] == 0)


def test_no_visit_above_energy_line(fbm_small):
    h, cells = fbm_small
    p = oracle.SimParams(mu=MU25, traj_per_cell=4, max_steps=500, seed=8)
    H, W = h.shape
    uphill = 0
    for c in cells[::7]:
        for j in range(p.traj_per_cell):
            tr = oracle.trace(h, 10.0, int(c), j, p)
            n = np.arange(tr["u"].size)
            z = fp64_paths.bilinear_f64(h, tr["u"], tr["v"])
            z0 = float(h.ravel()[c])
            # path length n D; e_n = z0 - z_n - mu n D up to FP32 rounding
            line = z0 - MU25 * 10.0 * n
            assert np.all(z <= line + 1e-2)
            assert np.allclose(tr["e"], z0 - z - MU25 * 10.0 * n, atol=2e-2)
            assert np.all(z[1:] < z0)
            dz = np.diff(z)
            de = np.diff(tr["e"].astype(np.float64))
            up = dz > 1e-3
            uphill += int(up.sum())
            assert np.all(de[up] < 0)
    assert uphill > 0


def test_drag_never_increases_energy_beyond_no_drag(fbm_small):
    h, cells = fbm_small
    a = oracle.SimParams(mu=MU25, traj_per_cell=4, max_steps=300, seed=4, randomness=0.0)
    b = oracle.SimParams(mu=MU25, traj_per_cell=4, max_steps=300, seed=4, randomness=0.0, drag_k=2e-3)
    _, ma, sa = oracle.simulate(h, 10.0, cells, a, "f64")
    _, mb, sb = oracle.simulate(h, 10.0, cells, b, "f64")
    assert sb["total_steps"] <= sa["total_steps"]
    assert np.all(mb <= ma + 1e-9)


def test_tiny_workload_sample_is_plausible():
    w = inputs.tiny()
    _, t2, _ = oracle.normals(w.dem_f32, w.cell_size)
    mask, cells = oracle.release(t2, 30.0, 45.0)
    assert 0.9 < mask.mean() < 1.0
    p = oracle.SimParams(mu=MU25, traj_per_cell=16, max_steps=1000, seed=0)
    c64, maxe, st = oracle.simulate(w.dem_f32, w.cell_size, cells[::97], p)
    assert c64.sum() == st["n_traj"] + st["total_steps"]
    vel = oracle.finalize(maxe)
    # 35-degree plane, 2.56 km fall: e <= 2560 m * (tan35 - tan25) + bump and gully relief
    assert 20.0 < vel.max() < math.sqrt(2 * 9.81 * (2560 * (math.tan(math.radians(35)) - MU25) + 300))
