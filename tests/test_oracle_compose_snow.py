"""Pins of the oracle's compose colouring (Sec. 3 / Fig. 4) and snow cover
(Sec. 5.1): exact stop colours, linear ramps, alpha-blend limits, and the
smoothstep closed form on planes."""
import math

import numpy as np
import pytest

import oracle
from paper_2506_23364_gb300 import inputs

STOPS = [(0.0, (0, 0, 0)), (10.0, (100, 200, 50)), (30.0, (255, 0, 255))]


def test_stop_colours_and_linear_ramp():
    v = np.array([-5.0, 0.0, 5.0, 10.0, 20.0, 30.0, 99.0], np.float32)
    cnt = np.ones(v.size, np.uint32)
    out = oracle.compose(v, cnt, STOPS, alpha=1.0, count_min=1)
    assert out[0, :3].tolist() == [0, 0, 0] and out[1, :3].tolist() == [0, 0, 0]
    assert out[2, :3].tolist() == [50, 100, 25]
    assert out[3, :3].tolist() == [100, 200, 50]
    assert out[4, :3].tolist() == [178, 100, 152]  # 100+77.5 -> 178 (half to even), 200-100, 50+102.5 -> 152
    assert out[5, :3].tolist() == [255, 0, 255] and out[6, :3].tolist() == [255, 0, 255]
    assert np.all(out[:, 3] == 255)


def test_alpha_and_blend_limits():
    rng = np.random.default_rng(1)
    v = rng.uniform(-3, 40, 500).astype(np.float32)
    cnt = rng.integers(0, 4, 500).astype(np.uint32)
    base = rng.integers(0, 256, (500, 4)).astype(np.uint8)
    o1 = oracle.compose(v, cnt, STOPS, alpha=1.0, count_min=2, base=base)
    plain = oracle.compose(v, cnt, STOPS, alpha=1.0, count_min=0)
    hit = cnt >= 2
    assert np.array_equal(o1[hit, :3], plain[hit, :3])
    assert np.array_equal(o1[~hit, :3], base[~hit, :3])
    assert np.array_equal(o1[:, 3], base[:, 3])
    o0 = oracle.compose(v, cnt, STOPS, alpha=0.0, count_min=0, base=base)
    assert np.array_equal(o0, base)
    half = oracle.compose(v, cnt, STOPS, alpha=0.5, count_min=0, base=base).astype(int)
    want = 0.5 * plain[:, :3].astype(float) + 0.5 * base[:, :3]
    assert np.all(np.abs(half[:, :3] - want) <= 0.5 + 1e-3)
    no_base = oracle.compose(v, cnt, STOPS, alpha=0.6, count_min=2)
    assert np.array_equal(no_base[:, 3], np.where(hit, 153, 0))


def _smooth(e0, e1, x):
    t = np.clip((x - e0) / (e1 - e0), 0, 1)
    return t * t * (3 - 2 * t)


@pytest.mark.parametrize("theta", [10.0, 29.0, 33.0, 45.0])
def test_snow_on_planes_closed_form(theta):
    cs = 5.0
    h = inputs.plane(30, 200, cs, math.tan(math.radians(theta)), 90.0, z0=2500.0, dtype=np.float64)
    nrm, _, _ = oracle.normals(h, cs, "f64")
    a, rgba = oracle.snow_cover(h, nrm[2], snow_line=2000.0, blend_alt=200.0, max_slope_deg=32.0,
                                blend_slope_deg=6.0, precision="f64")
    want = _smooth(1900.0, 2100.0, h) * _smooth(math.cos(math.radians(35.0)), math.cos(math.radians(29.0)),
                                                math.cos(math.radians(theta)))
    assert np.allclose(a, want, atol=1e-9)
    assert np.all(rgba[..., :3] == 255)
    assert np.array_equal(rgba[..., 3], np.rint(255 * a).astype(np.uint8))
    if theta <= 29.0:
        assert a.max() == 1.0  # flat enough and high enough: full snow
    if theta >= 35.0:
        assert a.max() == 0.0  # too steep everywhere


def test_snow_step_when_no_blend():
    h = np.array([[999.0, 1000.0, 1001.0]], np.float32)
    nz = np.ones_like(h)
    a, _ = oracle.snow_cover(h, nz, snow_line=1000.0, blend_alt=0.0, max_slope_deg=30.0, blend_slope_deg=0.0)
    assert a.tolist() == [[0.0, 1.0, 1.0]]
