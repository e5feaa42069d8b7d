"""Independent FP64 re-derivation of single avalanche trajectories (test code).

Written separately from the C oracle, in metres rather than cells, with the
bilinear height and gradient written as the weighted sum of the four corner
heights and the gradient divided by the cell size, as the trajectory reading
of Sec. 5.2 states them.  The Philox4x32-10 generator (Salmon et al., SC'11)
is a separate pure-Python implementation.  Used only to pin the oracle by
brute force on tiny grids.
"""
from __future__ import annotations

import math

import numpy as np

MASK = 0xFFFFFFFF


def philox_py(ctr, key):
    x = [c & MASK for c in ctr]
    k0, k1 = key[0] & MASK, key[1] & MASK
    for rnd in range(10):
        if rnd:
            k0 = (k0 + 0x9E3779B9) & MASK
            k1 = (k1 + 0xBB67AE85) & MASK
        a = 0xD2511F53 * x[0]
        b = 0xCD9E8D57 * x[2]
        x = [((b >> 32) ^ x[1] ^ k0) & MASK, b & MASK, ((a >> 32) ^ x[3] ^ k1) & MASK, a & MASK]
    return x


def uniforms(cell, j, n, seed):
    w = philox_py((cell, j, n // 2, 0), (seed & MASK, seed >> 32))
    a, b = (w[0], w[1]) if n % 2 == 0 else (w[2], w[3])
    return (a >> 8) / 2.0 ** 23 - 1.0, (b >> 8) / 2.0 ** 23 - 1.0


class Margin:
    """Smallest distance of any discrete decision from its threshold."""

    def __init__(self):
        self.m = math.inf

    def see(self, d):
        self.m = min(self.m, abs(d))


def _sample(h, cs, X, Y, mg: Margin):
    H, W = h.shape
    u = X / cs - 0.5
    v = Y / cs - 0.5
    i0 = math.floor(u)
    j0 = math.floor(v)
    if mg is not None:  # positions reached by a move; the start is exact
        mg.see(u - round(u))
        mg.see(v - round(v))
    fx = u - i0
    fy = v - j0
    i1 = min(i0 + 1, W - 1)
    j1 = min(j0 + 1, H - 1)
    h00, h10, h01, h11 = (float(h[j0, i0]), float(h[j0, i1]), float(h[j1, i0]), float(h[j1, i1]))
    z = (1 - fx) * (1 - fy) * h00 + fx * (1 - fy) * h10 + (1 - fx) * fy * h01 + fx * fy * h11
    dzdx = ((h10 - h00) * (1 - fy) + (h11 - h01) * fy) / cs
    dzdy = ((h01 - h00) * (1 - fx) + (h11 - h10) * fx) / cs
    return z, dzdx, dzdy


def _cell(W, cs, X, Y, mg):
    a, b = X / cs, Y / cs
    if mg is not None:
        mg.see(a - round(a))
        mg.see(b - round(b))
    return math.floor(b) * W + math.floor(a)


def path(h, cs, cell, j, *, mu, drag_k=0.0, persistence=0.9, randomness=0.16,
         step_scale=1.0, max_steps=64, seed=0, start=None):
    """Returns dict(X, Y, e, cell, end, margin) for trajectory (cell, j).
    ``cell`` keys the random stream; the start is the centre of that cell
    unless ``start`` gives it in metres (a release texel's centre)."""
    h = np.asarray(h, dtype=np.float64)
    H, W = h.shape
    mg = Margin()
    P, R = persistence, randomness
    D = step_scale * cs
    if start is None:
        X = (cell % W + 0.5) * cs
        Y = (cell // W + 0.5) * cs
    else:
        X, Y = float(start[0]), float(start[1])
    z, gx, gy = _sample(h, cs, X, Y, None)
    nrm = math.hypot(gx, gy)
    dx, dy = (-gx / nrm, -gy / nrm) if nrm > 0 else (0.0, 0.0)
    e = 0.0
    Xs, Ys, es, cells = [X], [Y], [e], [_cell(W, cs, X, Y, None)]
    end = "capped"
    for n in range(max_steps):
        z, gx, gy = _sample(h, cs, X, Y, None)
        nrm = math.hypot(gx, gy)
        if nrm > 0:
            ggx, ggy = -gx / nrm, -gy / nrm
        else:
            ggx, ggy = dx, dy
        xi_x, xi_y = uniforms(cell, j, n, seed)
        rx = P * dx + (1 - P) * ggx + R * xi_x
        ry = P * dy + (1 - P) * ggy + R * xi_y
        rn = math.hypot(rx, ry)
        if rn == 0:
            end = "stopped"
            break
        dx, dy = rx / rn, ry / rn
        X1 = X + D * dx
        Y1 = Y + D * dy
        u1, v1 = X1 / cs - 0.5, Y1 / cs - 0.5
        mg.see(u1)
        mg.see(u1 - (W - 1))
        mg.see(v1)
        mg.see(v1 - (H - 1))
        if not (0 <= u1 <= W - 1 and 0 <= v1 <= H - 1):
            end = "exited"
            break
        z1, _, _ = _sample(h, cs, X1, Y1, mg)
        e1 = e * (1 - drag_k * D) + (z - z1) - mu * D
        mg.see(e1 / max(1.0, abs(e)))
        if e1 <= 0:
            end = "stopped"
            break
        X, Y, e = X1, Y1, e1
        Xs.append(X)
        Ys.append(Y)
        es.append(e)
        cells.append(_cell(W, cs, X, Y, mg))
    return {"X": np.array(Xs), "Y": np.array(Ys), "e": np.array(es), "cell": np.array(cells),
            "end": end, "margin": mg.m}


def bilinear_f64(h, u, v):
    """FP64 bilinear height at cell-unit positions (arrays)."""
    h = np.asarray(h, dtype=np.float64)
    H, W = h.shape
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    i0 = np.floor(u).astype(np.int64)
    j0 = np.floor(v).astype(np.int64)
    i1 = np.minimum(i0 + 1, W - 1)
    j1 = np.minimum(j0 + 1, H - 1)
    fx = u - i0
    fy = v - j0
    return ((1 - fx) * (1 - fy) * h[j0, i0] + fx * (1 - fy) * h[j0, i1]
            + (1 - fx) * fy * h[j1, i0] + fx * fy * h[j1, i1])
