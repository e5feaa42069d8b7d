"""Pins of the oracle's release evaluation on a texture of chosen resolution
(Sec. 5.2: the user picks the texture resolution at which release points are
evaluated) and of particles started at release-texel centres.

Reading: the release texture covers the DEM's extent at 2^r times its
resolution; texel (a, b) is centred at ((a + 1/2) cs 2^-r, (b + 1/2) cs 2^-r)
in metres, clamped to the outermost cell centres; its steepness is the
bilinear interpolation of the cells' tan^2 there.  The pins below compute
texel centres in metres, interpolate with scipy, and check closed forms on
affine fields and planes.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2506_23364_gb300 import inputs
from tests import fp64_paths

MU25 = math.tan(math.radians(25.0))


def _centres_m(W, H, cs, r):
    """Texel centres in metres, written from the texture's extent (independent
    of the oracle's cell-unit formula)."""
    wr, hr = _dims(W, H, r)
    texel = cs * 2.0 ** (-r)
    X = np.clip((np.arange(wr) + 0.5) * texel, 0.5 * cs, (W - 0.5) * cs)
    Y = np.clip((np.arange(hr) + 0.5) * texel, 0.5 * cs, (H - 0.5) * cs)
    return X, Y


def _dims(W, H, r):
    if r >= 0:
        return W * 2 ** r, H * 2 ** r
    q = 2 ** (-r)
    return -(-W // q), -(-H // q)


@pytest.mark.parametrize("W,H", [(5, 3), (1, 1), (64, 17), (65536, 1)])
@pytest.mark.parametrize("r", [-3, -2, -1, 0, 1, 2, 3])
def test_dims(W, H, r):
    assert oracle.release_texture_dims(W, H, r) == _dims(W, H, r)


@pytest.mark.parametrize("r", [4, -4])
def test_dims_out_of_range(r):
    with pytest.raises(oracle.OracleError):
        oracle.release_texture_dims(8, 8, r)


def test_texture_too_large_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.release_texture_dims(65536, 8192, 1)  # 2^31 texels


@pytest.mark.parametrize("W,H,r,us,vs", [
    (4, 3, 1, [0, .25, .75, 1.25, 1.75, 2.25, 2.75, 3], [0, .25, .75, 1.25, 1.75, 2]),
    (5, 3, -1, [0.5, 2.5, 4], [0.5, 2]),
    (2, 1, 2, [0, 0, .125, .375, .625, .875, 1, 1], [0, 0, 0, 0]),
    (9, 2, -3, [3.5, 8], [1]),
])
def test_texel_centres_hand_computed(W, H, r, us, vs):
    """Start positions of particles (a trace with no move) at every texel."""
    h = np.linspace(0, 1, W * H).reshape(H, W).astype(np.float32)
    p = oracle.SimParams(max_steps=0, traj_per_cell=1, release_log2=r)
    wr, hr = oracle.release_texture_dims(W, H, r)
    assert (wr, hr) == (len(us), len(vs))
    for b in range(hr):
        for a in range(wr):
            tr = oracle.trace(h, 10.0, b * wr + a, 0, p)
            assert tr["u"][0] == np.float32(us[a]) and tr["v"][0] == np.float32(vs[b]), (a, b)
            assert tr["end"] == "capped" and tr["u"].size == 1


@pytest.mark.parametrize("seed", range(3))
def test_r0_equals_cell_release(seed):
    rng = np.random.default_rng(seed)
    t2 = rng.uniform(0, 2.0, size=(37, 53)).astype(np.float32)
    m0, c0 = oracle.release(t2, 30.0, 45.0)
    m1, c1 = oracle.release_texture(t2, 0, 30.0, 45.0)
    assert np.array_equal(m0, m1) and np.array_equal(c0, c1)


@pytest.mark.parametrize("r", [-2, -1, 1, 2, 3])
def test_affine_field_closed_form(r):
    """Bilinear interpolation reproduces an affine tan^2 field, so the release
    set is the set of texel centres where alpha + beta u + gamma v lies in
    range (FP64 build, decisions farther than 1e-9 from a bound)."""
    W, H = 29, 23
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    alpha, beta, gamma = 0.05, 0.031, 0.022
    t2 = alpha + beta * x + gamma * y
    lo, hi = 30.0, 45.0
    mask, tex = oracle.release_texture(t2, r, lo, hi, "f64")
    X, Y = _centres_m(W, H, 10.0, r)
    u = X / 10.0 - 0.5
    v = Y / 10.0 - 0.5
    T = alpha + beta * u[None, :] + gamma * v[:, None]
    t_lo, t_hi = math.tan(math.radians(lo)) ** 2, math.tan(math.radians(hi)) ** 2
    want = (T >= t_lo) & (T <= t_hi)
    clear = (np.abs(T - t_lo) > 1e-9) & (np.abs(T - t_hi) > 1e-9)
    assert clear.mean() > 0.95 and want.any() and (~want).any()
    assert np.array_equal(mask.astype(bool)[clear], want[clear])
    assert np.array_equal(tex, np.flatnonzero(mask.ravel()).astype(np.uint32))


@pytest.mark.parametrize("r", [-1, 1, 2])
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_random_field_vs_scipy(r, precision):
    """Independent interpolation (scipy, linear on the cell-centre lattice)
    at independently computed texel centres gives the same release set
    wherever the steepness is not within rounding of a bound."""
    interp = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(11 + r)
    W, H = 41, 27
    t2 = rng.uniform(0.1, 1.6, size=(H, W))
    t2 = t2.astype(np.float32 if precision == "f32" else np.float64)
    mask, _ = oracle.release_texture(t2, r, 30.0, 45.0, precision)
    X, Y = _centres_m(W, H, 10.0, r)
    f = interp.RegularGridInterpolator(((np.arange(H) + 0.5) * 10.0, (np.arange(W) + 0.5) * 10.0),
                                       t2.astype(np.float64), method="linear")
    YY, XX = np.meshgrid(Y, X, indexing="ij")
    T = f(np.stack([YY.ravel(), XX.ravel()], axis=1)).reshape(YY.shape)
    t_lo, t_hi = math.tan(math.radians(30.0)) ** 2, math.tan(math.radians(45.0)) ** 2
    want = (T >= t_lo) & (T <= t_hi)
    tol = 1e-5 if precision == "f32" else 1e-12
    clear = (np.abs(T - t_lo) > tol) & (np.abs(T - t_hi) > tol)
    assert clear.mean() > 0.99
    assert np.array_equal(mask.astype(bool)[clear], want[clear])


@pytest.mark.parametrize("r", [-3, -1, 1, 3])
def test_plane_releases_every_texel(r):
    cs = 10.0
    h = inputs.plane(40, 30, cs, math.tan(math.radians(35.0)), 90.0)
    _, t2, _ = oracle.normals(h.astype(np.float32), cs)
    mask, tex = oracle.release_texture(t2, r, 30.0, 45.0)
    assert mask.all() and tex.size == mask.size


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("r", [1, 2, -1])
def test_fall_line_from_texel(precision, r):
    """On a plane, with no random variation, a particle from a texel centre
    follows the fall line from that centre: u_n = u_0 + n, e_n = n D (tan - mu)."""
    cs, t = 10.0, math.tan(math.radians(35.0))
    W = H = 60
    dt = np.float32 if precision == "f32" else np.float64
    h = inputs.plane(W, H, cs, t, 0.0, z0=2000.0, dtype=dt)  # falls towards +x
    wr, hr = oracle.release_texture_dims(W, H, r)
    a, b = 3 * 2 ** max(r, 0) + 1, hr // 2 + 1
    X, Y = _centres_m(W, H, cs, r)
    u0, v0 = X[a] / cs - 0.5, Y[b] / cs - 0.5
    p = oracle.SimParams(mu=MU25, randomness=0.0, persistence=0.9, traj_per_cell=1, max_steps=500,
                         release_log2=r)
    tr = oracle.trace(h, cs, b * wr + a, 0, p, precision)
    n = np.arange(tr["u"].size)
    assert tr["end"] == "exited" and n.size > 40
    tol = 1e-9 if precision == "f64" else 2e-4
    assert np.allclose(tr["u"], u0 + n, atol=tol)
    assert np.allclose(tr["v"], v0, atol=tol)
    assert np.allclose(tr["e"], n * cs * (t - MU25), rtol=1e-5 if precision == "f32" else 1e-9,
                       atol=2e-3 if precision == "f32" else 1e-9)
    # visits: the cell containing each position, in metres
    cx = np.floor((tr["u"].astype(np.float64) + 0.5)).astype(np.int64)
    assert np.array_equal(tr["cell"], int(math.floor(Y[b] / cs)) * W + cx)


@pytest.mark.parametrize("seed", range(3))
def test_texel_paths_match_independent_fp64(seed):
    """Brute force: every particle of every texel of a small random grid
    equals the independent FP64 re-derivation started at the texel's centre
    in metres and keyed by the texel index."""
    rng = np.random.default_rng(300 + seed)
    W, H = int(rng.integers(6, 11)), int(rng.integers(6, 11))
    cs = 5.0
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    ang = rng.uniform(0, 2 * np.pi)
    h = 400.0 - 0.8 * cs * (x * np.cos(ang) + y * np.sin(ang)) + rng.normal(0, 0.1 * cs, size=(H, W))
    r = int(rng.choice([-1, 1, 2]))
    kw = dict(mu=float(rng.uniform(0.1, 0.5)), persistence=float(rng.uniform(0, 1)),
              randomness=float(rng.uniform(0, 0.4)), step_scale=float(rng.choice([1.0, 0.6])),
              max_steps=int(rng.integers(5, 40)), seed=int(rng.integers(0, 2 ** 63)))
    p = oracle.SimParams(traj_per_cell=2, release_log2=r, **kw)
    wr, hr = oracle.release_texture_dims(W, H, r)
    X, Y = _centres_m(W, H, cs, r)
    compared = 0
    for t in range(wr * hr):
        for j in range(2):
            ref = fp64_paths.path(h, cs, t, j, start=(X[t % wr], Y[t // wr]), **kw)
            if ref["margin"] < 1e-9:
                continue
            tr = oracle.trace(h, cs, t, j, p, "f64")
            assert tr["end"] == ref["end"], (t, j)
            assert np.allclose((tr["u"] + 0.5) * cs, ref["X"], atol=1e-9 * cs)
            assert np.allclose((tr["v"] + 0.5) * cs, ref["Y"], atol=1e-9 * cs)
            assert np.allclose(tr["e"], ref["e"], rtol=1e-9, atol=1e-9)
            assert np.array_equal(tr["cell"], ref["cell"])
            compared += 1
    assert compared > 0.8 * wr * hr * 2


def test_texel_raster_invariants_and_start_visits():
    rng = np.random.default_rng(5)
    W, H, cs = 31, 24, 10.0
    h = inputs.fbm(64, 0.8, seed=6, relief=500.0)[:H, :W].astype(np.float32)
    r = 2
    wr, hr = oracle.release_texture_dims(W, H, r)
    tex = np.sort(rng.choice(wr * hr, 200, replace=False)).astype(np.uint32)
    p = oracle.SimParams(mu=MU25, traj_per_cell=3, max_steps=200, seed=3, release_log2=r)
    c64, maxe, st = oracle.simulate(h, cs, tex, p)
    assert int(c64.sum()) == st["n_traj"] + st["total_steps"]
    assert st["n_traj"] == 600 == st["n_exited"] + st["n_capped"] + st["n_stopped"]
    # with no moves, the counts are the start visits: the cell containing each centre
    p0 = oracle.SimParams(traj_per_cell=3, max_steps=0, release_log2=r)
    c0, _, _ = oracle.simulate(h, cs, tex, p0)
    X, Y = _centres_m(W, H, cs, r)
    want = np.zeros(W * H, np.uint64)
    for t in tex:
        want[int(Y[t // wr] // cs) * W + int(X[t % wr] // cs)] += 3
    assert np.array_equal(c0.ravel(), want)


def test_texel_mode_rejections():
    h = np.zeros((8, 8), np.float32)
    with pytest.raises(oracle.OracleError):
        oracle.simulate(h, 1.0, np.array([16 * 16], np.uint32), oracle.SimParams(release_log2=1))
    oracle.simulate(h, 1.0, np.array([16 * 16 - 1], np.uint32), oracle.SimParams(release_log2=1, max_steps=3))
    with pytest.raises(oracle.OracleError):
        oracle.simulate(h, 1.0, np.array([0], np.uint32), oracle.SimParams(release_log2=4))
    with pytest.raises(oracle.OracleError):
        oracle.soft_forward(h, 1.0, np.array([0], np.uint32), np.ones(1), oracle.SimParams(release_log2=1))
