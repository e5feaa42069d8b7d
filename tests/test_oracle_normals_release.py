"""Pins of the oracle's normals, steepness and release selection (Sec. 5.2)."""
import numpy as np
import pytest

import oracle
from paper_2506_23364_gb300 import inputs


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("theta,azimuth", [(35.0, 90.0), (20.0, 30.0), (50.0, 200.0)])
def test_plane_gradient_closed_form(precision, theta, azimuth):
    cs = 10.0
    t = np.tan(np.deg2rad(theta))
    a = np.deg2rad(azimuth)
    dt = np.float32 if precision == "f32" else np.float64
    h = inputs.plane(40, 33, cs, t, azimuth, z0=3000.0, dtype=dt)
    nrm, t2, sd = oracle.normals(h, cs, precision)
    gx_true, gy_true = -t * np.cos(a), -t * np.sin(a)
    # exact plane: central and one-sided differences both give the slope
    tol = 2e-4 if precision == "f32" else 1e-10  # FP32 heights near 3000 m carry ~1e-4 m rounding
    nx_true = -gx_true / np.sqrt(1 + t * t)
    ny_true = -gy_true / np.sqrt(1 + t * t)
    nz_true = 1 / np.sqrt(1 + t * t)
    assert np.allclose(nrm[0], nx_true, atol=tol)
    assert np.allclose(nrm[1], ny_true, atol=tol)
    assert np.allclose(nrm[2], nz_true, atol=tol)
    assert np.allclose(t2, t * t, rtol=tol * 4)
    assert np.allclose(sd, theta, atol=50 * tol)


def test_normals_match_numpy_gradient_fp64():
    # np.gradient: central differences inside, first-order one-sided at the edges
    rng = np.random.default_rng(3)
    h = rng.uniform(0, 500, size=(37, 53))
    cs = 7.5
    nrm, t2, sd = oracle.normals(h, cs, "f64")
    gy, gx = np.gradient(h, cs, edge_order=1)
    assert np.allclose(t2, gx * gx + gy * gy, rtol=1e-12, atol=1e-12)
    L = np.sqrt(1 + gx * gx + gy * gy)
    assert np.allclose(nrm[0], -gx / L, rtol=1e-12, atol=1e-14)
    assert np.allclose(nrm[1], -gy / L, rtol=1e-12, atol=1e-14)
    assert np.allclose(nrm[2], 1 / L, rtol=1e-12)
    assert np.allclose(sd, np.degrees(np.arctan(np.hypot(gx, gy))), rtol=1e-12)
    assert np.allclose((nrm ** 2).sum(axis=0), 1.0, rtol=1e-14)


def test_single_row_and_column_have_zero_derivative_across():
    h = np.arange(7, dtype=np.float64)[None, :] * 3.0
    nrm, t2, _ = oracle.normals(h, 1.0, "f64")
    assert np.allclose(t2, 9.0)
    assert np.all(nrm[1] == 0)
    h1 = np.arange(5, dtype=np.float64)[:, None] * 2.0
    nrm, t2, _ = oracle.normals(h1, 1.0, "f64")
    assert np.allclose(t2, 4.0)
    assert np.all(nrm[0] == 0)
    nrm, t2, _ = oracle.normals(np.array([[5.0]]), 1.0, "f64")
    assert t2[0, 0] == 0 and nrm[2, 0, 0] == 1


def test_release_plane_35_all_cells_selected():
    h = inputs.plane(64, 48, 10.0, np.tan(np.deg2rad(35.0)))
    _, t2, _ = oracle.normals(h, 10.0)
    mask, cells = oracle.release(t2, 30.0, 45.0)
    assert mask.all() and cells.size == 64 * 48
    mask, cells = oracle.release(t2, 36.0, 45.0)
    assert not mask.any() and cells.size == 0


def test_release_range_inclusive_and_sorted():
    lo, hi = 30.0, 45.0
    tlo = oracle.tan2_threshold(lo)
    thi = oracle.tan2_threshold(hi)
    vals = np.array([np.nextafter(tlo, np.float32(0)), tlo, np.nextafter(tlo, np.float32(9)),
                     np.nextafter(thi, np.float32(0)), thi, np.nextafter(thi, np.float32(9)),
                     np.float32(0), np.float32(np.inf)], dtype=np.float32)
    t2 = np.tile(vals, (3, 1))
    mask, cells = oracle.release(t2, lo, hi)
    assert mask[0].tolist() == [0, 1, 1, 1, 1, 0, 0, 0]
    assert np.array_equal(cells, np.flatnonzero(mask.ravel()).astype(np.uint32))


def test_release_random_matches_definition():
    rng = np.random.default_rng(11)
    t2 = rng.uniform(0, 2, size=(57, 91)).astype(np.float32)
    mask, cells = oracle.release(t2, 20.0, 40.0)
    want = (t2 >= oracle.tan2_threshold(20.0)) & (t2 <= oracle.tan2_threshold(40.0))
    assert np.array_equal(mask.astype(bool), want)
    assert np.array_equal(cells, np.flatnonzero(want.ravel()))
    assert np.all(np.diff(cells.astype(np.int64)) > 0)


@pytest.mark.parametrize("lo,hi", [(-1.0, 10.0), (40.0, 30.0), (10.0, 90.0)])
def test_release_rejects_bad_range(lo, hi):
    with pytest.raises(oracle.OracleError) as ei:
        oracle.release(np.zeros((4, 4), np.float32), lo, hi)
    assert ei.value.code == 1


def test_decode_is_one_float_multiply():
    q = np.array([0, 1, 7, 12345, 30000, 65535], dtype=np.uint16)
    h = oracle.decode_u16(q, 0.1)
    assert np.array_equal(h, q.astype(np.float32) * np.float32(0.1))
