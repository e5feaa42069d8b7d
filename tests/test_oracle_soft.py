"""Pins of the oracle's soft-deposit mode and its FP64 reverse-mode gradient.

* mass: every particle deposits exactly its weight;
* closed form on an inclined plane with no random variation: e_m =
  m D (tan(theta) - mu), S_m = prod sigma(e_i / tau), deposits w (S_{m-1} - S_m)
  down the fall line and the rest at the exit row; d/dmu in closed form;
* the reverse-mode gradient equals central finite differences of the loss
  L = sum (D - D*)^2 in log-parameters and in the release weights.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2506_23364_gb300 import inputs

MU25 = math.tan(math.radians(25.0))


def _sig(x):
    return 1.0 / (1.0 + np.exp(-x))


def test_mass_is_conserved():
    z = inputs.fbm(64, 0.8, seed=3, relief=600.0).astype(np.float32)
    _, t2, _ = oracle.normals(z, 10.0)
    _, cells = oracle.release(t2, 30.0, 45.0)
    w = np.random.default_rng(0).uniform(0.5, 1.5, cells.size)
    p = oracle.SimParams(mu=MU25, drag_k=1e-3, traj_per_cell=8, max_steps=300, seed=1)
    D, st = oracle.soft_forward(z, 10.0, cells, w, p)
    assert st["n_traj"] == 8 * cells.size
    assert abs(D.sum() - 8 * w.sum()) < 1e-9 * D.sum()
    assert np.all(D >= 0)


@pytest.mark.parametrize("mu_scale", [0.6, 1.3])
def test_plane_closed_form_deposits_and_mu_derivative(mu_scale):
    cs, t = 10.0, math.tan(math.radians(30.0))
    W, H = 7, 60
    h = inputs.plane(W, H, cs, t, 90.0, z0=3000.0, dtype=np.float64)  # FP64 build: no height rounding
    mu = MU25 * mu_scale
    p = oracle.SimParams(mu=mu, drag_k=0.0, randomness=0.0, persistence=0.9, traj_per_cell=1, max_steps=1000)
    cells = np.array([3], np.uint32)  # row 0, column 3
    w = np.array([1.25])
    D, st = oracle.soft_forward(h, cs, cells, w, p, precision="f64")
    Dd = cs  # one cell per move
    m = np.arange(1, H)
    e = m * Dd * (t - mu)
    S = np.concatenate([[1.0], np.cumprod(_sig(e / oracle.SOFT_TAU))])
    cut = np.nonzero(S < 1e-7)[0]
    n = int(cut[0]) if cut.size else H - 1
    col = np.zeros(H)
    col[1:n + 1] = w[0] * (S[:n] - S[1:n + 1])
    col[n] += w[0] * S[n]
    assert np.allclose(D[:, 3], col, rtol=1e-9, atol=1e-12)
    assert np.all(D[:, [0, 1, 2, 4, 5, 6]] == 0)
    # d/dlog mu of J = sum G D with G = row index (closed form by the product rule)
    G = np.broadcast_to(np.arange(H, dtype=np.float64)[:, None], (H, W)).copy()
    gth, gw = oracle.soft_gradient(h, cs, cells, w, p, G, precision="f64")
    de = -m[:n] * Dd  # de_m/dmu
    sig = _sig(e[:n] / oracle.SOFT_TAU)
    dlogS = np.cumsum((1.0 - sig) * de / oracle.SOFT_TAU)  # d log S_m / dmu
    dS = np.concatenate([[0.0], S[1:n + 1] * dlogS])
    rows = np.arange(H)
    dJ = w[0] * (np.sum(rows[1:n + 1] * (dS[:n] - dS[1:n + 1])) + rows[n] * dS[n])
    assert abs(gth[0] - mu * dJ) <= 1e-8 * max(1.0, abs(mu * dJ))
    J = np.sum(G * D)
    assert abs(gw[0] - J / w[0]) <= 1e-9 * abs(J)


def _loss(z, cs, cells, w, p, Dstar):
    D, _ = oracle.soft_forward(z, cs, cells, w, p)
    return np.sum((D - Dstar) ** 2), D


def test_reverse_gradient_matches_central_differences():
    z = inputs.fbm(48, 0.8, seed=11, relief=500.0, m=56).astype(np.float32)
    _, t2, _ = oracle.normals(z, 10.0)
    _, cells = oracle.release(t2, 30.0, 50.0)
    cells = cells[::3]
    rng = np.random.default_rng(4)
    w = rng.uniform(0.5, 1.5, cells.size)
    base = dict(persistence=0.8, randomness=0.2, traj_per_cell=6, max_steps=400, seed=9)
    mu0, k0 = MU25, 1e-3
    pstar = oracle.SimParams(mu=mu0 * 1.2, drag_k=k0 * 0.8, **base)
    Dstar, _ = oracle.soft_forward(z, 10.0, cells, w, pstar)
    p0 = oracle.SimParams(mu=mu0, drag_k=k0, **base)
    L0, D0 = _loss(z, 10.0, cells, w, p0, Dstar)
    gth, gw = oracle.soft_gradient(z, 10.0, cells, w, p0, 2.0 * (D0 - Dstar))
    hh = 1e-4
    for i, (name, val) in enumerate((("mu", mu0), ("drag_k", k0))):
        lp = _loss(z, 10.0, cells, w, oracle.SimParams(**{**base, "mu": mu0, "drag_k": k0, name: val * math.exp(hh)}),
                   Dstar)[0]
        lm = _loss(z, 10.0, cells, w, oracle.SimParams(**{**base, "mu": mu0, "drag_k": k0, name: val * math.exp(-hh)}),
                   Dstar)[0]
        fd = (lp - lm) / (2 * hh)
        assert abs(gth[i] - fd) <= 2e-4 * abs(fd) + 1e-9, (name, gth[i], fd)
    for c in (0, cells.size // 2, cells.size - 1):
        wp, wm = w.copy(), w.copy()
        wp[c] += 1e-5
        wm[c] -= 1e-5
        fd = (_loss(z, 10.0, cells, wp, p0, Dstar)[0] - _loss(z, 10.0, cells, wm, p0, Dstar)[0]) / 2e-5
        assert abs(gw[c] - fd) <= 1e-5 * max(1.0, abs(fd)), (c, gw[c], fd)
