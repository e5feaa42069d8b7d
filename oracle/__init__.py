"""CPU oracle of the avalanche-overlay hot path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``awo_oracle.c`` (plain C,
compiled in FP32 and in FP64 with contraction off) through ctypes and shares no
code with the CUDA library.

Every function follows the paper's description of the avalanche workflow
(Sec. 5.2) and overlay mipmap (Sec. 3); see the C source for the step-by-step
reading.  ``precision`` selects the FP32 build (the parity oracle) or the FP64
build (for closed-form pins).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_LIBS: dict[str, ctypes.CDLL] = {}

_U32P = ctypes.POINTER(ctypes.c_uint32)


def _real(precision: str):
    return (ctypes.c_float, np.float32) if precision == "f32" else (ctypes.c_double, np.float64)


def _params_type(precision: str):
    creal, _ = _real(precision)

    class Params(ctypes.Structure):
        _fields_ = [("mu", creal), ("drag_k", creal), ("persistence", creal),
                    ("randomness", creal), ("step_scale", creal), ("gravity", creal),
                    ("traj_per_cell", ctypes.c_uint32), ("max_steps", ctypes.c_uint32),
                    ("seed", ctypes.c_uint64), ("release_log2", ctypes.c_int32)]
    return Params


class Stats(ctypes.Structure):
    _fields_ = [("total_steps", ctypes.c_uint64), ("n_traj", ctypes.c_uint64),
                ("n_exited", ctypes.c_uint64), ("n_capped", ctypes.c_uint64),
                ("n_stopped", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_PARAMS = {p: _params_type(p) for p in ("f32", "f64")}


def lib(precision: str = "f32") -> ctypes.CDLL:
    if precision not in _LIBS:
        path = _build.lib_path(precision)
        if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_build.SRC):
            _build.build()
        L = ctypes.CDLL(path)
        L.orc_real_size.restype = ctypes.c_int
        want = 4 if precision == "f32" else 8
        if L.orc_real_size() != want:
            raise RuntimeError(f"oracle {path} computes in {L.orc_real_size()}-byte reals, expected {want}")
        _LIBS[precision] = L
    return _LIBS[precision]


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: status {code}")
        self.code = code


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(rc, what)


# ----------------------------------------------------------------------------
# Philox4x32-10
# ----------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> tuple[int, int, int, int]:
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib("f32").orc_philox4x32_10(c, k, o)
    return tuple(int(x) for x in o)


def draw(cell: int, j: int, n: int, seed: int, precision: str = "f32") -> tuple[float, float]:
    """The two uniforms in [-1, 1) that move n of trajectory (cell, j) uses."""
    creal, npr = _real(precision)
    xi = (creal * 2)()
    lib(precision).orc_draw(ctypes.c_uint32(cell), ctypes.c_uint32(j), ctypes.c_uint32(n),
                            ctypes.c_uint64(seed), xi)
    return npr(xi[0]), npr(xi[1])


def draws(cell: int, j: int, n_moves: int, seed: int, precision: str = "f32") -> np.ndarray:
    return np.array([draw(cell, j, n, seed, precision) for n in range(n_moves)])


# ----------------------------------------------------------------------------
# Stages
# ----------------------------------------------------------------------------
def decode_u16(q: np.ndarray, scale: float = 0.1, precision: str = "f32") -> np.ndarray:
    creal, npr = _real(precision)
    q = np.ascontiguousarray(q, dtype=np.uint16)
    h = np.empty(q.shape, dtype=npr)
    lib(precision).orc_decode_u16(_ptr(q), ctypes.c_int64(q.size), creal(scale), _ptr(h))
    return h


def normals(h: np.ndarray, cs: float, precision: str = "f32", want_slope: bool = True):
    """Returns (nrm[3,H,W], tan2[H,W], slope_deg[H,W] or None)."""
    creal, npr = _real(precision)
    h = np.ascontiguousarray(h, dtype=npr)
    H, W = h.shape
    nrm = np.empty((3, H, W), dtype=npr)
    t2 = np.empty((H, W), dtype=npr)
    sd = np.empty((H, W), dtype=npr) if want_slope else None
    rc = lib(precision).orc_normals(_ptr(h), ctypes.c_int32(W), ctypes.c_int32(H), creal(cs),
                                    _ptr(nrm), _ptr(t2), _ptr(sd))
    _check(rc, "orc_normals")
    return nrm, t2, sd


def release(tan2: np.ndarray, lo_deg: float, hi_deg: float, precision: str = "f32"):
    """Returns (mask[H,W] uint8, cells uint32 sorted)."""
    _, npr = _real(precision)
    t2 = np.ascontiguousarray(tan2, dtype=npr)
    H, W = t2.shape
    mask = np.empty((H, W), dtype=np.uint8)
    cells = np.empty(W * H, dtype=np.uint32)
    n = ctypes.c_uint32(0)
    rc = lib(precision).orc_release(_ptr(t2), ctypes.c_int32(W), ctypes.c_int32(H),
                                    ctypes.c_double(lo_deg), ctypes.c_double(hi_deg),
                                    _ptr(mask), _ptr(cells), ctypes.byref(n))
    _check(rc, "orc_release")
    return mask, cells[: n.value].copy()


def release_texture_dims(W: int, H: int, r: int) -> tuple[int, int]:
    """(Wr, Hr) of the release texture at 2^r times the DEM's resolution."""
    wr, hr = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = lib("f32").orc_release_texture_dims(ctypes.c_int32(W), ctypes.c_int32(H), ctypes.c_int32(r),
                                             ctypes.byref(wr), ctypes.byref(hr))
    _check(rc, "orc_release_texture_dims")
    return int(wr.value), int(hr.value)


def release_texture(tan2: np.ndarray, r: int, lo_deg: float, hi_deg: float, precision: str = "f32"):
    """Release points on the texture at 2^r times the DEM's resolution:
    (mask[Hr, Wr] uint8, texel indices uint32 sorted)."""
    _, npr = _real(precision)
    t2 = np.ascontiguousarray(tan2, dtype=npr)
    H, W = t2.shape
    wr, hr = release_texture_dims(W, H, r)
    mask = np.empty((hr, wr), dtype=np.uint8)
    texels = np.empty(wr * hr, dtype=np.uint32)
    n = ctypes.c_uint32(0)
    rc = lib(precision).orc_release_texture(_ptr(t2), ctypes.c_int32(W), ctypes.c_int32(H), ctypes.c_int32(r),
                                            ctypes.c_double(lo_deg), ctypes.c_double(hi_deg),
                                            _ptr(mask), _ptr(texels), ctypes.byref(n))
    _check(rc, "orc_release_texture")
    return mask, texels[: n.value].copy()


@dataclass
class SimParams:
    mu: float = 0.46630765815499864  # tan(25 deg)
    drag_k: float = 0.0
    persistence: float = 0.9
    randomness: float = 0.16
    step_scale: float = 1.0
    gravity: float = 9.81
    traj_per_cell: int = 16
    max_steps: int = 1000
    seed: int = 0
    release_log2: int = 0  # list entries are texels of the release texture at 2^r x the DEM resolution

    def to_c(self, precision: str):
        return _PARAMS[precision](self.mu, self.drag_k, self.persistence, self.randomness,
                                  self.step_scale, self.gravity, self.traj_per_cell,
                                  self.max_steps, self.seed, self.release_log2)


def simulate(h: np.ndarray, cs: float, cells: np.ndarray, params: SimParams,
             precision: str = "f32", count64: np.ndarray | None = None,
             maxe: np.ndarray | None = None):
    """Accumulates into (count64 uint64[H,W], maxe real[H,W]); returns them and stats."""
    creal, npr = _real(precision)
    h = np.ascontiguousarray(h, dtype=npr)
    H, W = h.shape
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    if count64 is None:
        count64 = np.zeros((H, W), dtype=np.uint64)
    if maxe is None:
        maxe = np.zeros((H, W), dtype=npr)
    st = Stats()
    p = params.to_c(precision)
    rc = lib(precision).orc_simulate(_ptr(h), ctypes.c_int32(W), ctypes.c_int32(H), creal(cs),
                                     _ptr(cells), ctypes.c_uint32(cells.size), ctypes.byref(p),
                                     _ptr(count64), _ptr(maxe), ctypes.byref(st))
    _check(rc, "orc_simulate")
    return count64, maxe, st.as_dict()


def counts_u32(count64: np.ndarray) -> np.ndarray:
    """Count raster as uint32; raises OracleError(5) where a cell exceeds 2^32-1."""
    if count64.size and int(count64.max()) > 0xFFFFFFFF:
        raise OracleError(5, "count overflow")
    return count64.astype(np.uint32)


END_NAMES = {0: "capped", 1: "exited", 2: "stopped"}


def trace(h: np.ndarray, cs: float, cell: int, j: int, params: SimParams,
          precision: str = "f32", cap: int | None = None) -> dict:
    creal, npr = _real(precision)
    h = np.ascontiguousarray(h, dtype=npr)
    H, W = h.shape
    cap = cap if cap is not None else params.max_steps + 1
    u = np.empty(cap, dtype=npr)
    v = np.empty(cap, dtype=npr)
    e = np.empty(cap, dtype=npr)
    c = np.empty(cap, dtype=np.int64)
    n = ctypes.c_int64(0)
    end = ctypes.c_int32(0)
    p = params.to_c(precision)
    rc = lib(precision).orc_trace(_ptr(h), ctypes.c_int32(W), ctypes.c_int32(H), creal(cs),
                                  ctypes.c_uint32(cell), ctypes.c_uint32(j), ctypes.byref(p),
                                  ctypes.c_int64(cap), _ptr(u), _ptr(v), _ptr(e), _ptr(c),
                                  ctypes.byref(n), ctypes.byref(end))
    _check(rc, "orc_trace")
    k = n.value
    return {"u": u[:k].copy(), "v": v[:k].copy(), "e": e[:k].copy(), "cell": c[:k].copy(),
            "end": END_NAMES[end.value]}


SOFT_TAU = 1.0  # metres of energy-line height per e-fold of survival


def soft_forward(h: np.ndarray, cs: float, cells: np.ndarray, weights: np.ndarray, params: SimParams,
                 tau: float = SOFT_TAU, precision: str = "f32", threads: int = 1):
    """Soft deposits (FP64 raster [H, W]) of every particle; weights per release entry."""
    from concurrent.futures import ThreadPoolExecutor

    creal, npr = _real(precision)
    h = np.ascontiguousarray(h, dtype=npr)
    H, W = h.shape
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    weights = np.ascontiguousarray(weights, dtype=np.float64)
    p = params.to_c(precision)
    parts = [(c, w) for c, w in zip(np.array_split(cells, threads), np.array_split(weights, threads)) if c.size] \
        or [(cells, weights)]

    def one(cw):
        c, w = cw
        dep = np.zeros((H, W), np.float64)
        st = Stats()
        rc = lib(precision).orc_soft_forward(_ptr(h), ctypes.c_int32(W), ctypes.c_int32(H), creal(cs), _ptr(c),
                                             ctypes.c_uint32(c.size), _ptr(w), ctypes.byref(p),
                                             ctypes.c_double(tau), _ptr(dep), ctypes.byref(st))
        _check(rc, "orc_soft_forward")
        return dep, st.as_dict()

    with ThreadPoolExecutor(len(parts)) as ex:
        out = list(ex.map(one, parts))
    dep = out[0][0]
    for d, _ in out[1:]:
        dep += d
    stats = {k: sum(o[1][k] for o in out) for k in out[0][1]}
    return dep, stats


def soft_gradient(h: np.ndarray, cs: float, cells: np.ndarray, weights: np.ndarray, params: SimParams,
                  G: np.ndarray, tau: float = SOFT_TAU, precision: str = "f32", threads: int = 1,
                  with_abs: bool = False):
    """FP64 reverse-mode gradient of sum(G * D): (d/dlog mu, d/dlog k), d/dw per release entry;
    with_abs: also the sums over particles of |each particle's (d/dlog mu, d/dlog k) term|."""
    from concurrent.futures import ThreadPoolExecutor

    creal, npr = _real(precision)
    h = np.ascontiguousarray(h, dtype=npr)
    H, W = h.shape
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    weights = np.ascontiguousarray(weights, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    p = params.to_c(precision)
    idx = [i for i in np.array_split(np.arange(cells.size), threads) if i.size] or [np.arange(0)]

    def one(ix):
        c = np.ascontiguousarray(cells[ix])
        w = np.ascontiguousarray(weights[ix])
        gt = np.zeros(2, np.float64)
        ga = np.zeros(2, np.float64)
        gw = np.zeros(c.size, np.float64)
        rc = lib(precision).orc_soft_gradient(_ptr(h), ctypes.c_int32(W), ctypes.c_int32(H), creal(cs), _ptr(c),
                                              ctypes.c_uint32(c.size), _ptr(w), ctypes.byref(p),
                                              ctypes.c_double(tau), _ptr(G), _ptr(gt), _ptr(gw), _ptr(ga))
        _check(rc, "orc_soft_gradient")
        return ix, gt, gw, ga

    with ThreadPoolExecutor(len(idx)) as ex:
        out = list(ex.map(one, idx))
    gtheta = np.zeros(2, np.float64)
    gabs = np.zeros(2, np.float64)
    gw = np.zeros(cells.size, np.float64)
    for ix, gt, g, ga in out:
        gtheta += gt
        gabs += ga
        gw[ix] = g
    return (gtheta, gw, gabs) if with_abs else (gtheta, gw)


def finalize(maxe: np.ndarray, gravity: float = 9.81, precision: str = "f32") -> np.ndarray:
    creal, npr = _real(precision)
    m = np.ascontiguousarray(maxe, dtype=npr)
    vel = np.empty_like(m)
    lib(precision).orc_finalize(_ptr(m), ctypes.c_int64(m.size), creal(gravity), _ptr(vel))
    return vel


def lod(count: np.ndarray, vel: np.ndarray, levels: int, precision: str = "f32"):
    """Returns lists of count and vel rasters for levels 0..levels-1 (level 0 = inputs)."""
    _, npr = _real(precision)
    count = np.ascontiguousarray(count, dtype=np.uint32)
    vel = np.ascontiguousarray(vel, dtype=npr)
    H, W = count.shape
    cs_out, vs_out = [], []
    w, hh = W, H
    for _ in range(1, levels):
        w, hh = (w + 1) // 2, (hh + 1) // 2
        cs_out.append(np.empty((hh, w), dtype=np.uint32))
        vs_out.append(np.empty((hh, w), dtype=npr))
    n = max(levels - 1, 1)
    cp = (ctypes.c_void_p * n)(*[a.ctypes.data for a in cs_out] or [None])
    vp = (ctypes.c_void_p * n)(*[a.ctypes.data for a in vs_out] or [None])
    rc = lib(precision).orc_lod(_ptr(count), _ptr(vel), ctypes.c_int32(W), ctypes.c_int32(H),
                                ctypes.c_int32(levels), cp, vp)
    _check(rc, "orc_lod")
    return [count] + cs_out, [vel] + vs_out


def tan2_threshold(deg: float, precision: str = "f32") -> float:
    """tan^2 of an angle in degrees, computed in FP64 and rounded once."""
    _, npr = _real(precision)
    t = np.tan(np.float64(deg) * (np.pi / 180.0))
    return npr(t * t)


def overlay(h: np.ndarray, cs: float, lo_deg: float, hi_deg: float, params: SimParams,
            levels: int = 1, precision: str = "f32") -> dict:
    """The whole workflow: normals -> release -> simulate -> velocity -> mipmap."""
    nrm, t2, sd = normals(h, cs, precision)
    mask, cells = release(t2, lo_deg, hi_deg, precision)
    c64, maxe, st = simulate(h, cs, cells, params, precision)
    count = counts_u32(c64)
    vel = finalize(maxe, params.gravity, precision)
    cl, vl = lod(count, vel, levels, precision)
    return {"normals": nrm, "tan2": t2, "slope_deg": sd, "mask": mask, "cells": cells,
            "count": count, "maxe": maxe, "vel": vel, "count_lv": cl, "vel_lv": vl, "stats": st}


def simulate_threaded(h: np.ndarray, cs: float, cells: np.ndarray, params: SimParams, threads: int | None = None,
                      precision: str = "f32", merge: bool = True):
    """orc_simulate over contiguous chunks of the release list on `threads`
    host threads (ctypes drops the GIL), each into private rasters; the
    rasters are merged by sum (counts) and max (energy), which is exactly the
    single-thread result because both reductions are order-independent."""
    from concurrent.futures import ThreadPoolExecutor

    threads = max(1, int(threads or os.cpu_count() or 1))
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    chunks = [c for c in np.array_split(cells, threads) if c.size] or [cells]
    _, npr = _real(precision)
    h = np.ascontiguousarray(h, dtype=npr)

    def one(c):
        return simulate(h, cs, c, params, precision,
                        count64=np.zeros(h.shape, np.uint64), maxe=np.zeros(h.shape, npr))

    with ThreadPoolExecutor(len(chunks)) as ex:
        parts = list(ex.map(one, chunks))
    stats = {k: sum(p[2][k] for p in parts) for k in parts[0][2]}
    if not merge:
        return None, None, stats
    count64, maxe = parts[0][0], parts[0][1]
    for c, m, _ in parts[1:]:
        count64 += c
        np.maximum(maxe, m, out=maxe)
    return count64, maxe, stats



# ----------------------------------------------------------------------------
# Compose and snow cover
# ----------------------------------------------------------------------------
class _Colormap(ctypes.Structure):
    _fields_ = [("n_stops", ctypes.c_int32), ("value", ctypes.c_float * 16), ("rgb", (ctypes.c_uint8 * 3) * 16),
                ("pad", ctypes.c_uint8 * 4), ("alpha", ctypes.c_float), ("count_min", ctypes.c_uint32)]


def compose(value: np.ndarray, count: np.ndarray, stops, alpha: float, count_min: int, base: np.ndarray | None = None,
            precision: str = "f32") -> np.ndarray:
    """RGBA8 [..., 4] overlay colouring and alpha blend (see awo_oracle.c)."""
    _, npr = _real(precision)
    v = np.ascontiguousarray(value, dtype=npr)
    c = np.ascontiguousarray(count, dtype=np.uint32)
    cm = _Colormap()
    cm.n_stops = len(stops)
    for i, (x, rgb) in enumerate(stops):
        cm.value[i] = float(x)
        for k in range(3):
            cm.rgb[i][k] = int(rgb[k])
    cm.alpha = float(alpha)
    cm.count_min = int(count_min)
    out = np.empty(v.shape + (4,), np.uint8)
    b = None if base is None else np.ascontiguousarray(base, dtype=np.uint8)
    rc = lib(precision).orc_compose(_ptr(v), _ptr(c), ctypes.c_int64(v.size), ctypes.byref(cm), _ptr(b), _ptr(out))
    _check(rc, "orc_compose")
    return out


def snow_cover(h: np.ndarray, nz: np.ndarray, snow_line: float, blend_alt: float, max_slope_deg: float,
               blend_slope_deg: float, precision: str = "f32"):
    """(alpha [H, W], RGBA8 [H, W, 4]) of the snow-cover overlay (see awo_oracle.c)."""
    _, npr = _real(precision)
    hh = np.ascontiguousarray(h, dtype=npr)
    z = np.ascontiguousarray(nz, dtype=npr)
    a = np.empty(hh.shape, npr)
    rgba = np.empty(hh.shape + (4,), np.uint8)
    rc = lib(precision).orc_snow_cover(_ptr(hh), _ptr(z), ctypes.c_int64(hh.size), ctypes.c_double(snow_line),
                                       ctypes.c_double(blend_alt), ctypes.c_double(max_slope_deg),
                                       ctypes.c_double(blend_slope_deg), _ptr(a), _ptr(rgba))
    _check(rc, "orc_snow_cover")
    return a, rgba
