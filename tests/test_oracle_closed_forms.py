"""Closed-form pins of the oracle's trajectory model (Sec. 5.2 reading).

On an inclined plane with no random variation, a particle follows the straight
fall line and its energy-line height after n moves of horizontal length D is
n D (tan(theta) - mu) (no drag), or ((tan(theta) - mu) / k)(1 - (1 - k D)^n)
with drag k.  On a plane running into a flat, the particle stops where the
energy line meets the terrain: at horizontal distance L tan(theta) / mu from
release.  These follow from the runout-angle criterion alone.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2506_23364_gb300 import inputs

MU25 = math.tan(math.radians(25.0))


def _params(**kw):
    base = dict(mu=MU25, drag_k=0.0, persistence=0.9, randomness=0.0, step_scale=1.0,
                gravity=9.81, traj_per_cell=1, max_steps=1000, seed=0)
    base.update(kw)
    return oracle.SimParams(**base)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("azimuth", [90.0, 0.0, 33.0, 121.0])
@pytest.mark.parametrize("drag_k", [0.0, 1e-3])
def test_straight_fall_line(precision, azimuth, drag_k):
    cs, theta = 10.0, 35.0
    t = math.tan(math.radians(theta))
    W = H = 120
    dt = np.float32 if precision == "f32" else np.float64
    h = inputs.plane(W, H, cs, t, azimuth, z0=3000.0, dtype=dt)
    a = math.radians(azimuth)
    x0 = 60 - int(round(50 * math.cos(a)))
    y0 = 60 - int(round(50 * math.sin(a)))
    cell = y0 * W + x0
    p = _params(drag_k=drag_k, persistence=0.9)
    tr = oracle.trace(h, cs, cell, 0, p, precision)
    n = np.arange(tr["u"].size)
    assert tr["end"] == "exited"
    assert n.size > 50
    D = cs
    if drag_k == 0:
        e_true = n * D * (t - MU25)
    else:
        e_true = ((t - MU25) / drag_k) * (1 - (1 - drag_k * D) ** n)
    if precision == "f64":
        assert np.allclose(tr["u"], x0 + n * math.cos(a), atol=1e-9)
        assert np.allclose(tr["v"], y0 + n * math.sin(a), atol=1e-9)
        assert np.allclose(tr["e"], e_true, rtol=1e-9, atol=1e-9)
    else:
        assert np.allclose(tr["u"], x0 + n * math.cos(a), atol=2e-4)
        assert np.allclose(tr["v"], y0 + n * math.sin(a), atol=2e-4)
        assert np.allclose(tr["e"], e_true, rtol=1e-5, atol=2e-3)
    # recorded cells: nearest cell centre of each position
    cx = np.floor(tr["u"].astype(np.float64) + 0.5).astype(np.int64)
    cy = np.floor(tr["v"].astype(np.float64) + 0.5).astype(np.int64)
    assert np.array_equal(tr["cell"], cy * W + cx)


def test_fall_line_velocity_raster():
    cs, t = 10.0, math.tan(math.radians(35.0))
    W, H = 9, 200
    h = inputs.plane(W, H, cs, t, 90.0, z0=3000.0, dtype=np.float64)
    p = _params(traj_per_cell=3)
    cells = np.array([4], dtype=np.uint32)  # row 0, column 4
    c64, maxe, st = oracle.simulate(h, cs, cells, p, "f64")
    vel = oracle.finalize(maxe, 9.81, "f64")
    rows = np.arange(H)
    # every row of column 4 visited by all three identical trajectories
    assert np.array_equal(c64[:, 4], np.full(H, 3))
    assert c64.sum() == 3 * H
    assert np.allclose(vel[:, 4], np.sqrt(2 * 9.81 * rows * cs * (t - MU25)), rtol=1e-9)
    assert st == {"total_steps": 3 * (H - 1), "n_traj": 3, "n_exited": 3, "n_capped": 0, "n_stopped": 0}


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("L", [30, 50, 77])
def test_runout_on_flat(precision, L):
    cs, t = 10.0, math.tan(math.radians(35.0))
    W, H = 11, 400
    dt = np.float32 if precision == "f32" else np.float64
    h = inputs.plane_to_flat(W, H, cs, t, L, z0=3000.0, dtype=dt)
    tr = oracle.trace(h, cs, 5, 0, _params(), precision)
    v_star = L * t / MU25  # energy line meets the flat
    assert abs(v_star - round(v_star)) > 1e-3
    assert tr["end"] == "stopped"
    assert float(tr["v"][-1]) == math.floor(v_star)
    runout_on_flat = float(tr["v"][-1]) - L
    assert abs(runout_on_flat - (L * t / MU25 - L)) < 1.0


def test_slope_below_runout_angle_stops_at_once():
    cs = 10.0
    h = inputs.plane(20, 20, cs, math.tan(math.radians(20.0)), 90.0)
    p = _params(randomness=0.16, traj_per_cell=8)
    cells = np.arange(0, 20 * 19, 7, dtype=np.uint32)
    c64, maxe, st = oracle.simulate(h, cs, cells, p)
    # border cells may step out of the domain first; no move is ever recorded
    assert st["total_steps"] == 0 and st["n_stopped"] + st["n_exited"] == st["n_traj"] == 8 * cells.size
    assert st["n_stopped"] > 0.8 * st["n_traj"]
    assert c64.sum() == st["n_traj"] and np.all(maxe == 0)


def test_energy_tie_stops():
    # cs = 1, heights drop exactly 0.5 per row, mu D = 0.5: e_1 = 0 exactly -> stop
    h = (100.0 - 0.5 * np.arange(12, dtype=np.float32))[:, None].repeat(5, axis=1).astype(np.float32)
    tr = oracle.trace(h, 1.0, 2, 0, _params(mu=0.5, persistence=0.9, randomness=0.0))
    assert tr["end"] == "stopped" and tr["u"].size == 1
    tr = oracle.trace(h, 1.0, 2, 0, _params(mu=0.25, persistence=0.9, randomness=0.0))
    assert tr["end"] == "exited" and tr["u"].size == 12
    assert np.array_equal(tr["e"], 0.25 * np.arange(12, dtype=np.float32))
    assert np.array_equal(tr["v"], np.arange(12, dtype=np.float32))


def test_cap_and_zero_cap():
    h = inputs.plane(10, 300, 10.0, math.tan(math.radians(40.0)), 90.0)
    tr = oracle.trace(h, 10.0, 4, 0, _params(max_steps=5))
    assert tr["end"] == "capped" and tr["u"].size == 6
    tr = oracle.trace(h, 10.0, 4, 0, _params(max_steps=0))
    assert tr["end"] == "capped" and tr["u"].size == 1
    c64, maxe, st = oracle.simulate(h, 10.0, np.array([4, 5], np.uint32), _params(max_steps=0, traj_per_cell=2))
    assert st["n_capped"] == 4 and st["total_steps"] == 0 and c64.sum() == 4


def test_full_persistence_keeps_initial_direction():
    # P = 1, R = 0: the direction never changes, even on curved terrain
    w = inputs.tiny()
    h = w.dem_f32.astype(np.float64)
    cell = 40 * 256 + 100
    tr = oracle.trace(h, 10.0, cell, 0, _params(persistence=1.0), "f64")
    assert tr["u"].size > 20
    du, dv = np.diff(tr["u"]), np.diff(tr["v"])
    assert np.allclose(du, du[0], atol=1e-12) and np.allclose(dv, dv[0], atol=1e-12)
    assert abs(du[0] ** 2 + dv[0] ** 2 - 1) < 1e-12


def test_flat_start_without_randomness_stops():
    h = np.full((6, 6), 100.0)
    tr = oracle.trace(h, 10.0, 14, 0, _params(randomness=0.0), "f64")
    assert tr["end"] == "stopped" and tr["u"].size == 1


@pytest.mark.parametrize("kw", [dict(persistence=1.5), dict(randomness=-0.1), dict(mu=-1.0),
                                dict(drag_k=0.2), dict(step_scale=0.0), dict(step_scale=1.5)])
def test_invalid_parameters_rejected(kw):
    h = np.zeros((4, 4), np.float32)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.simulate(h, 10.0, np.array([0], np.uint32), _params(**kw))
    assert ei.value.code == 1


def test_release_cell_out_of_range_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.simulate(np.zeros((4, 4), np.float32), 10.0, np.array([16], np.uint32), _params())
