"""Brute-force pin: the FP64 oracle's trajectories equal an independent FP64
re-derivation (tests/fp64_paths.py, written in metres) on small random grids,
wherever no discrete decision lies within 1e-9 of its threshold."""
import math

import numpy as np
import pytest

import oracle
from tests import fp64_paths

MU25 = math.tan(math.radians(25.0))


def _grid(rng, W, H, cs):
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    tilt = rng.uniform(0.5, 1.0) * cs
    ang = rng.uniform(0, 2 * np.pi)
    z = 500.0 - tilt * (x * np.cos(ang) + y * np.sin(ang)) + rng.normal(0, 0.15 * cs, size=(H, W))
    return z


@pytest.mark.parametrize("seed", range(6))
def test_paths_match_independent_fp64(seed):
    rng = np.random.default_rng(100 + seed)
    W, H = int(rng.integers(8, 17)), int(rng.integers(8, 17))
    cs = float(rng.choice([1.0, 5.0, 10.0]))
    h = _grid(rng, W, H, cs)
    kw = dict(mu=float(rng.uniform(0.1, 0.6)), drag_k=float(rng.choice([0.0, 0.01 / cs])),
              persistence=float(rng.uniform(0, 1)), randomness=float(rng.uniform(0, 0.5)),
              step_scale=float(rng.choice([1.0, 0.5, 0.73])), max_steps=int(rng.integers(1, 65)),
              seed=int(rng.integers(0, 2 ** 63)))
    p = oracle.SimParams(traj_per_cell=4, gravity=9.81, **kw)
    compared = 0
    moves = 0
    for cell in range(W * H):
        for j in range(4):
            ref = fp64_paths.path(h, cs, cell, j, **kw)
            if ref["margin"] < 1e-9:
                continue
            tr = oracle.trace(h, cs, cell, j, p, "f64")
            assert tr["end"] == ref["end"], (cell, j)
            assert tr["u"].size == ref["X"].size, (cell, j)
            assert np.allclose((tr["u"] + 0.5) * cs, ref["X"], atol=1e-9 * cs)
            assert np.allclose((tr["v"] + 0.5) * cs, ref["Y"], atol=1e-9 * cs)
            assert np.allclose(tr["e"], ref["e"], rtol=1e-9, atol=1e-9)
            assert np.array_equal(tr["cell"], ref["cell"])
            compared += 1
            moves += tr["u"].size - 1
    assert compared > 0.9 * W * H * 4
    assert moves > 0


def test_raster_is_aggregate_of_paths():
    """count and max-energy rasters equal the visits of all traced paths."""
    rng = np.random.default_rng(7)
    W, H, cs = 23, 19, 10.0
    h = _grid(rng, W, H, cs).astype(np.float32)
    p = oracle.SimParams(mu=MU25, persistence=0.8, randomness=0.3, traj_per_cell=5, max_steps=40, seed=99)
    cells = np.arange(0, W * H, 3, dtype=np.uint32)
    c64, maxe, st = oracle.simulate(h, cs, cells, p)
    cnt = np.zeros(W * H, np.uint64)
    mx = np.zeros(W * H, np.float32)
    steps = 0
    for c in cells:
        for j in range(p.traj_per_cell):
            tr = oracle.trace(h, cs, int(c), j, p)
            np.add.at(cnt, tr["cell"], 1)
            np.maximum.at(mx, tr["cell"], tr["e"])
            steps += tr["u"].size - 1
    assert np.array_equal(c64.ravel(), cnt)
    assert np.array_equal(maxe.ravel(), mx)
    assert st["total_steps"] == steps
    assert c64.sum() == st["n_traj"] + st["total_steps"]
