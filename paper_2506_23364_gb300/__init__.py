"""GB300 avalanche-overlay hot path: Python binding of ``libawo.so``.

The functions below carry the names of the C ABI in ``include/awo.h`` and do
argument marshalling only: they check tensor dtypes, devices and sizes, pass
raw device pointers and the current CUDA stream to the library, and raise
``AwoError`` on a non-OK status.  Every step of the computation runs in the
library's CUDA kernels; there is no fallback.  PyTorch supplies device memory
and streams.

Importing the package does not load the library; the first call does, and it
raises ``RuntimeError`` when ``libawo.so`` is missing (build it with
``python -c "import __graft_entry__ as g; g.build()"``).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libawo.so")

AWO_OK, AWO_EINVAL, AWO_ENOMEM, AWO_ECUDA, AWO_ETIMEOUT, AWO_EOVERFLOW, AWO_ECANCELLED = range(7)


class AwoError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


class Grid(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("cell_size", ctypes.c_float)]

    def __repr__(self):
        return f"Grid({self.width}x{self.height}, {self.cell_size} m)"

    @property
    def cells(self) -> int:
        return int(self.width) * int(self.height)


class SimParams(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_float), ("drag_k", ctypes.c_float), ("persistence", ctypes.c_float),
                ("randomness", ctypes.c_float), ("step_scale", ctypes.c_float), ("gravity", ctypes.c_float),
                ("traj_per_cell", ctypes.c_uint32), ("max_steps", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("flags", ctypes.c_uint32), ("release_log2", ctypes.c_int32)]

    @classmethod
    def make(cls, mu=math.tan(math.radians(25.0)), drag_k=0.0, persistence=0.9, randomness=0.16,
             step_scale=1.0, gravity=9.81, traj_per_cell=16, max_steps=1000, seed=0, flags=0, release_log2=0):
        return cls(mu, drag_k, persistence, randomness, step_scale, gravity, traj_per_cell, max_steps,
                   seed, flags, release_log2)


class SimRequest(ctypes.Structure):
    """awo_sim_request: one region of a batched particle launch."""
    _fields_ = [("d_h", ctypes.c_void_p), ("grid", Grid), ("d_cells", ctypes.c_void_p),
                ("d_n_cells", ctypes.c_void_p), ("n_cells_max", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("params", SimParams), ("d_count", ctypes.c_void_p), ("d_maxe", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    """awo_tuning: launch shape of the batched particle kernel."""
    _fields_ = [("threads_per_block", ctypes.c_int32), ("group_particles", ctypes.c_int32),
                ("refill", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"threads_per_block": int(self.threads_per_block), "group_particles": int(self.group_particles),
                "refill": "warp" if self.refill == REFILL_WARP else "lane"}


class Colormap(ctypes.Structure):
    """awo_colormap: colour ramp (up to 16 stops) and overlay opacity."""
    _fields_ = [("n_stops", ctypes.c_int32), ("value", ctypes.c_float * 16), ("rgb", (ctypes.c_uint8 * 3) * 16),
                ("pad", ctypes.c_uint8 * 4), ("alpha", ctypes.c_float), ("count_min", ctypes.c_uint32)]

    @classmethod
    def make(cls, stops, alpha: float = 0.75, count_min: int = 1):
        """stops: [(value, (r, g, b)), ...] with increasing values."""
        cm = cls()
        cm.n_stops = len(stops)
        for i, (v, c) in enumerate(stops):
            cm.value[i] = float(v)
            for k in range(3):
                cm.rgb[i][k] = int(c[k])
        cm.alpha = float(alpha)
        cm.count_min = int(count_min)
        return cm


# Velocity colour scale for the overlay (m/s): blue -> cyan -> green -> yellow -> red.
VELOCITY_STOPS = [(0.0, (40, 40, 200)), (10.0, (0, 190, 230)), (25.0, (40, 200, 60)), (45.0, (250, 220, 0)),
                  (70.0, (220, 30, 30))]


class SnowParams(ctypes.Structure):
    _fields_ = [("snow_line_m", ctypes.c_float), ("blend_alt_m", ctypes.c_float),
                ("max_slope_deg", ctypes.c_float), ("blend_slope_deg", ctypes.c_float)]


REFILL_LANE, REFILL_WARP = 0, 1
BATCH_MAX = 128
STATS_FIELDS = ("total_steps", "n_traj", "n_exited", "n_capped", "n_stopped", "n_rejected")

_lib = None


def lib() -> ctypes.CDLL:
    """Loads libawo.so (once) and declares the C prototypes."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: the CUDA library must be built (there is no CPU path)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, u32, f32, f64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_float,
                                  ctypes.c_double, ctypes.c_size_t)
    st = ctypes.c_int
    protos = {
        "awo_status_string": (ctypes.c_char_p, [st]),
        "awo_version": (i32, []),
        "awo_decode_u16": (st, [vp, Grid, f32, vp, vp]),
        "awo_normals": (st, [vp, Grid, vp, vp, vp, vp]),
        "awo_release_workspace_bytes": (sz, [Grid]),
        "awo_release": (st, [vp, Grid, f64, f64, vp, vp, vp, vp, sz, vp]),
        "awo_release_noalloc": (st, [vp, Grid, f64, f64, vp, vp, vp, vp]),
        "awo_release_from_mask": (st, [vp, Grid, vp, vp, vp, sz, vp]),
        "awo_release_texture_dims": (st, [Grid, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "awo_release_texture_workspace_bytes": (sz, [Grid, i32]),
        "awo_release_texture": (st, [vp, Grid, i32, f64, f64, vp, vp, vp, vp, sz, vp]),
        "awo_simulate_workspace_bytes": (sz, [u32]),
        "awo_dem_gather_path": (st, [vp, Grid, vp, ctypes.POINTER(i32)]),
        "awo_simulate": (st, [vp, Grid, vp, vp, u32, ctypes.POINTER(SimParams), vp, vp, vp, vp, sz, vp]),
        "awo_finalize": (st, [vp, Grid, f32, vp, vp]),
        "awo_normals_u16": (st, [vp, Grid, f32, vp, vp, vp, vp, vp]),
        "awo_overlay_lod": (st, [vp, vp, Grid, i32, vp, vp, vp]),
        "awo_finalize_lod": (st, [vp, vp, Grid, f32, i32, vp, vp, vp, vp]),
        "awo_simulate_batched_workspace_bytes": (sz, [vp, i32]),
        "awo_simulate_batched": (st, [vp, i32, vp, vp, vp, sz, vp]),
        "awo_tune_batched": (st, [vp, i32, vp, sz, vp, vp, vp]),
        "awo_soft_workspace_bytes": (sz, [u32]),
        "awo_soft_forward": (st, [vp, Grid, vp, vp, u32, vp, ctypes.POINTER(SimParams), f32, vp, vp, vp, sz, vp]),
        "awo_soft_backward": (st, [vp, Grid, vp, vp, u32, vp, ctypes.POINTER(SimParams), f32, vp, vp, vp, vp, sz,
                                   vp]),
        "awo_fixed_to_real": (st, [vp, ctypes.c_int64, vp, vp]),
        "awo_compose": (st, [vp, vp, Grid, ctypes.POINTER(Colormap), vp, vp, vp]),
        "awo_snow_cover": (st, [vp, vp, Grid, ctypes.POINTER(SnowParams), vp, vp, vp]),
        "awo_probe_l2_gather": (st, [vp, u32, u32, vp, vp]),
        "awo_probe_l2_red": (st, [vp, u32, u32, vp]),
        "awo_probe_threads": (ctypes.c_uint64, []),
        "awo_selftest_rcp_sqrt": (st, [u32, ctypes.c_uint64, vp, vp]),
        "awo_selftest_visit_cell": (st, [u32, ctypes.c_uint64, vp, vp]),
        "awo_selftest_div_rn": (st, [vp, u32, u32, vp, vp]),
        "awo_simulate_time_kernel": (st, [vp, vp]),
        "awo_probe_philox": (st, [vp, ctypes.c_int64, ctypes.c_uint64, i32, vp, vp]),
    }
    for name, (res, args) in protos.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def status_string(status: int) -> str:
    return lib().awo_status_string(status).decode()


def _check(status: int, what: str):
    if status != AWO_OK:
        raise AwoError(status, what)


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dev(t: torch.Tensor | None, dtype, numel: int | None, name: str):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {numel}")
    return t.data_ptr()


def grid(width: int, height: int, cell_size: float) -> Grid:
    return Grid(int(width), int(height), float(cell_size))


# ----------------------------------------------------------------------------
# The C ABI, one function each
# ----------------------------------------------------------------------------
def awo_decode_u16(q: torch.Tensor, g: Grid, scale: float, h: torch.Tensor, stream=None):
    """q: uint16 heights (an int16 tensor holding the same bits is accepted)."""
    if q.dtype not in (torch.uint16, torch.int16):
        raise TypeError("q must be uint16 (or int16 bits)")
    _check(lib().awo_decode_u16(_dev(q, q.dtype, g.cells, "q"), g, scale,
                                _dev(h, torch.float32, g.cells, "h"), _stream(stream)), "awo_decode_u16")


def awo_normals(h: torch.Tensor, g: Grid, normal=None, tan2=None, slope_deg=None, stream=None):
    n = g.cells
    _check(lib().awo_normals(_dev(h, torch.float32, n, "h"), g, _dev(normal, torch.float32, 3 * n, "normal"),
                             _dev(tan2, torch.float32, n, "tan2"), _dev(slope_deg, torch.float32, n, "slope_deg"),
                             _stream(stream)), "awo_normals")


def awo_normals_u16(q: torch.Tensor, g: Grid, scale: float, h: torch.Tensor, normal=None, tan2=None, slope_deg=None,
                    stream=None):
    """awo_decode_u16 then awo_normals in one pass (see awo.h)."""
    if q.dtype not in (torch.uint16, torch.int16):
        raise TypeError("q must be uint16 (or int16 bits)")
    n = g.cells
    _check(lib().awo_normals_u16(_dev(q, q.dtype, n, "q"), g, scale, _dev(h, torch.float32, n, "h"),
                                 _dev(normal, torch.float32, 3 * n, "normal"), _dev(tan2, torch.float32, n, "tan2"),
                                 _dev(slope_deg, torch.float32, n, "slope_deg"), _stream(stream)), "awo_normals_u16")


def awo_release_workspace_bytes(g: Grid) -> int:
    return int(lib().awo_release_workspace_bytes(g))


def awo_release(tan2: torch.Tensor, g: Grid, slope_lo_deg: float, slope_hi_deg: float, mask, cells: torch.Tensor,
                n: torch.Tensor, ws: torch.Tensor, stream=None):
    c = g.cells
    if cells.dtype not in (torch.int32, torch.uint32) or n.dtype not in (torch.int32, torch.uint32):
        raise TypeError("cells and n must be int32 or uint32")
    _check(lib().awo_release(_dev(tan2, torch.float32, c, "tan2"), g, slope_lo_deg, slope_hi_deg,
                             _dev(mask, torch.uint8, c, "mask"), _dev(cells, cells.dtype, c, "cells"),
                             _dev(n, n.dtype, 1, "n"), _dev(ws, torch.uint8, None, "ws"), ws.numel(),
                             _stream(stream)), "awo_release")


def awo_release_from_mask(mask: torch.Tensor, g: Grid, cells: torch.Tensor, n: torch.Tensor, ws: torch.Tensor,
                          stream=None):
    """Ordered release list from a caller's uint8 mask (known release areas)."""
    c = g.cells
    if cells.dtype not in (torch.int32, torch.uint32) or n.dtype not in (torch.int32, torch.uint32):
        raise TypeError("cells and n must be int32 or uint32")
    _check(lib().awo_release_from_mask(_dev(mask, torch.uint8, c, "mask"), g, _dev(cells, cells.dtype, c, "cells"),
                                       _dev(n, n.dtype, 1, "n"), _dev(ws, torch.uint8, None, "ws"), ws.numel(),
                                       _stream(stream)), "awo_release_from_mask")


RELEASE_LOG2_MAX = 3


def awo_release_texture_dims(g: Grid, release_log2: int) -> tuple[int, int]:
    """(Wr, Hr) of the release texture at 2^release_log2 times the DEM resolution."""
    w, h = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(lib().awo_release_texture_dims(g, int(release_log2), ctypes.byref(w), ctypes.byref(h)),
           "awo_release_texture_dims")
    return int(w.value), int(h.value)


def awo_release_texture_workspace_bytes(g: Grid, release_log2: int) -> int:
    return int(lib().awo_release_texture_workspace_bytes(g, int(release_log2)))


def awo_release_texture(tan2: torch.Tensor, g: Grid, release_log2: int, slope_lo_deg: float, slope_hi_deg: float,
                        mask: torch.Tensor, texels: torch.Tensor, n: torch.Tensor, ws: torch.Tensor, stream=None):
    """Release points on the texture at 2^release_log2 times the DEM resolution:
    mask [Hr, Wr] uint8 and the ordered texel indices."""
    wr, hr = awo_release_texture_dims(g, release_log2)
    t = wr * hr
    if texels.dtype not in (torch.int32, torch.uint32) or n.dtype not in (torch.int32, torch.uint32):
        raise TypeError("texels and n must be int32 or uint32")
    _check(lib().awo_release_texture(_dev(tan2, torch.float32, g.cells, "tan2"), g, int(release_log2),
                                     slope_lo_deg, slope_hi_deg, _dev(mask, torch.uint8, t, "mask"),
                                     _dev(texels, texels.dtype, t, "texels"), _dev(n, n.dtype, 1, "n"),
                                     _dev(ws, torch.uint8, None, "ws"), ws.numel(), _stream(stream)),
           "awo_release_texture")


RELEASE_NOALLOC_MAX_CELLS = 8192 * 8192


def awo_release_noalloc(tan2: torch.Tensor, g: Grid, slope_lo_deg: float, slope_hi_deg: float, mask,
                        cells: torch.Tensor, n: torch.Tensor, stream=None):
    """awo_release without a workspace, for callers that cannot hand the
    library extra device memory (a plug-in whose host application owns the
    device allocator, a real-time loop that allocates nothing after start-up).
    The scratch is a fixed 128 KiB array inside the library; grids above
    RELEASE_NOALLOC_MAX_CELLS cells are refused, and calls that overlap on the
    GPU race on the shared array."""
    c = g.cells
    if c > RELEASE_NOALLOC_MAX_CELLS:
        raise AwoError(AWO_ENOMEM, f"awo_release_noalloc: grid of {c} cells exceeds the built-in scratch "
                                   f"limit of {RELEASE_NOALLOC_MAX_CELLS} cells (8192 x 8192)")
    if cells.dtype not in (torch.int32, torch.uint32) or n.dtype not in (torch.int32, torch.uint32):
        raise TypeError("cells and n must be int32 or uint32")
    _check(lib().awo_release_noalloc(_dev(tan2, torch.float32, c, "tan2"), g, slope_lo_deg, slope_hi_deg,
                                     _dev(mask, torch.uint8, c, "mask"), _dev(cells, cells.dtype, c, "cells"),
                                     _dev(n, n.dtype, 1, "n"), _stream(stream)), "awo_release_noalloc")


def awo_dem_gather_path(h: torch.Tensor, g: Grid, stream=None) -> str:
    """'texture' or 'loads': how the particle kernels fetch this DEM buffer's footprints."""
    t = ctypes.c_int32(0)
    _check(lib().awo_dem_gather_path(_dev(h, torch.float32, g.cells, "h"), g, _stream(stream), ctypes.byref(t)),
           "awo_dem_gather_path")
    return "texture" if t.value else "loads"


def awo_simulate_workspace_bytes(n_cells_max: int) -> int:
    return int(lib().awo_simulate_workspace_bytes(int(n_cells_max)))


def awo_simulate(h: torch.Tensor, g: Grid, cells: torch.Tensor | None, n_cells_dev: torch.Tensor | None,
                 n_cells_max: int, params: SimParams, count: torch.Tensor, maxe: torch.Tensor,
                 stats: torch.Tensor | None, ws: torch.Tensor, stream=None):
    c = g.cells
    cells_ptr = None
    if cells is not None:
        cells_ptr = _dev(cells, cells.dtype, n_cells_max, "cells")
        if cells.dtype not in (torch.int32, torch.uint32):
            raise TypeError("cells must be int32 or uint32")
    ndev = _dev(n_cells_dev, n_cells_dev.dtype, 1, "n_cells_dev") if n_cells_dev is not None else None
    if count.dtype not in (torch.int32, torch.uint32):
        raise TypeError("count must be int32 or uint32")
    count_ptr = _dev(count, count.dtype, c, "count")
    sp = _dev(stats, torch.int64, 6, "stats") if stats is not None else None
    _check(lib().awo_simulate(_dev(h, torch.float32, c, "h"), g, cells_ptr, ndev, int(n_cells_max),
                              ctypes.byref(params), count_ptr, _dev(maxe, torch.float32, c, "maxe"), sp,
                              _dev(ws, torch.uint8, None, "ws"), ws.numel(), _stream(stream)), "awo_simulate")


def sim_request(h: torch.Tensor, g: Grid, cells: torch.Tensor | None, n_cells_dev: torch.Tensor | None,
                n_cells_max: int, params: SimParams, count: torch.Tensor, maxe: torch.Tensor) -> SimRequest:
    """Checks the tensors of one region and packs them as an awo_sim_request."""
    c = g.cells
    if count.dtype not in (torch.int32, torch.uint32):
        raise TypeError("count must be int32 or uint32")
    cp = None
    if cells is not None:
        if cells.dtype not in (torch.int32, torch.uint32):
            raise TypeError("cells must be int32 or uint32")
        cp = _dev(cells, cells.dtype, n_cells_max, "cells")
    nd = _dev(n_cells_dev, n_cells_dev.dtype, 1, "n_cells_dev") if n_cells_dev is not None else None
    return SimRequest(_dev(h, torch.float32, c, "h"), g, cp, nd, int(n_cells_max), 0, params,
                      _dev(count, count.dtype, c, "count"), _dev(maxe, torch.float32, c, "maxe"))


def _req_array(reqs):
    if isinstance(reqs, ctypes.Array):
        return reqs
    arr = (SimRequest * len(reqs))()
    for i, r in enumerate(reqs):
        arr[i] = r
    return arr


def awo_simulate_batched_workspace_bytes(reqs) -> int:
    arr = _req_array(reqs)
    n = int(lib().awo_simulate_batched_workspace_bytes(arr, len(arr)))
    if n == 0:
        raise AwoError(AWO_EINVAL, "awo_simulate_batched_workspace_bytes")
    return n


def awo_simulate_batched(reqs, ws: torch.Tensor, tuning: Tuning | None = None, stats: torch.Tensor | None = None,
                         stream=None):
    """One persistent launch over all regions; stats: int64 [n_req, 6] on the device."""
    arr = _req_array(reqs)
    sp = _dev(stats, torch.int64, 6 * len(arr), "stats") if stats is not None else None
    _check(lib().awo_simulate_batched(arr, len(arr), ctypes.byref(tuning) if tuning is not None else None, sp,
                                      _dev(ws, torch.uint8, None, "ws"), ws.numel(), _stream(stream)),
           "awo_simulate_batched")


def awo_tune_batched(reqs, ws: torch.Tensor, stream=None) -> tuple[Tuning, float]:
    arr = _req_array(reqs)
    best = Tuning()
    ms = ctypes.c_float(0.0)
    _check(lib().awo_tune_batched(arr, len(arr), _dev(ws, torch.uint8, None, "ws"), ws.numel(), _stream(stream),
                                  ctypes.byref(best), ctypes.byref(ms)), "awo_tune_batched")
    return best, float(ms.value)


def awo_soft_workspace_bytes(n_cells_max: int) -> int:
    return int(lib().awo_soft_workspace_bytes(int(n_cells_max)))


def _cells_args(cells, n_cells_dev, n_cells_max):
    cp = None
    if cells is not None:
        if cells.dtype not in (torch.int32, torch.uint32):
            raise TypeError("cells must be int32 or uint32")
        cp = _dev(cells, cells.dtype, n_cells_max, "cells")
    nd = _dev(n_cells_dev, n_cells_dev.dtype, 1, "n_cells_dev") if n_cells_dev is not None else None
    return cp, nd


def awo_soft_forward(h: torch.Tensor, g: Grid, cells, n_cells_dev, n_cells_max: int, weight: torch.Tensor,
                     params: SimParams, tau: float, deposit: torch.Tensor, stats: torch.Tensor | None,
                     ws: torch.Tensor, stream=None):
    """Soft deposits (int64 fixed point, 2^-32) of every particle; see awo.h."""
    cp, nd = _cells_args(cells, n_cells_dev, n_cells_max)
    _check(lib().awo_soft_forward(_dev(h, torch.float32, g.cells, "h"), g, cp, nd, int(n_cells_max),
                                  _dev(weight, torch.float32, n_cells_max, "weight"), ctypes.byref(params),
                                  float(tau), _dev(deposit, torch.int64, g.cells, "deposit"),
                                  _dev(stats, torch.int64, 6, "stats") if stats is not None else None,
                                  _dev(ws, torch.uint8, None, "ws"), ws.numel(), _stream(stream)), "awo_soft_forward")


def awo_soft_backward(h: torch.Tensor, g: Grid, cells, n_cells_dev, n_cells_max: int, weight: torch.Tensor,
                      params: SimParams, tau: float, grad_deposit: torch.Tensor, grad_theta: torch.Tensor,
                      grad_weight: torch.Tensor, ws: torch.Tensor, stream=None):
    """dL/dlog(mu), dL/dlog(k) (FP64 [2]) and dL/dw (FP32 per release entry) given dL/dD."""
    cp, nd = _cells_args(cells, n_cells_dev, n_cells_max)
    _check(lib().awo_soft_backward(_dev(h, torch.float32, g.cells, "h"), g, cp, nd, int(n_cells_max),
                                   _dev(weight, torch.float32, n_cells_max, "weight"), ctypes.byref(params),
                                   float(tau), _dev(grad_deposit, torch.float32, g.cells, "grad_deposit"),
                                   _dev(grad_theta, torch.float64, 2, "grad_theta"),
                                   _dev(grad_weight, torch.float32, n_cells_max, "grad_weight"),
                                   _dev(ws, torch.uint8, None, "ws"), ws.numel(), _stream(stream)),
           "awo_soft_backward")


def awo_fixed_to_real(q: torch.Tensor, out: torch.Tensor, stream=None):
    _check(lib().awo_fixed_to_real(_dev(q, torch.int64, None, "q"), q.numel(),
                                   _dev(out, torch.float64, q.numel(), "out"), _stream(stream)), "awo_fixed_to_real")


def awo_compose(value: torch.Tensor, count: torch.Tensor, g: Grid, cm: Colormap, base_rgba: torch.Tensor | None,
                out_rgba: torch.Tensor, stream=None):
    """Colour-mapped overlay (RGBA8 [H, W, 4]), alpha-blended over base_rgba when given."""
    c = g.cells
    if count.dtype not in (torch.int32, torch.uint32):
        raise TypeError("count must be int32 or uint32")
    _check(lib().awo_compose(_dev(value, torch.float32, c, "value"), _dev(count, count.dtype, c, "count"), g,
                             ctypes.byref(cm), _dev(base_rgba, torch.uint8, 4 * c, "base_rgba"),
                             _dev(out_rgba, torch.uint8, 4 * c, "out_rgba"), _stream(stream)), "awo_compose")


def awo_snow_cover(h: torch.Tensor, nz: torch.Tensor, g: Grid, p: SnowParams, alpha: torch.Tensor | None = None,
                   rgba: torch.Tensor | None = None, stream=None):
    c = g.cells
    _check(lib().awo_snow_cover(_dev(h, torch.float32, c, "h"), _dev(nz, torch.float32, c, "nz"), g, ctypes.byref(p),
                                _dev(alpha, torch.float32, c, "alpha"), _dev(rgba, torch.uint8, 4 * c, "rgba"),
                                _stream(stream)), "awo_snow_cover")


def awo_finalize(maxe: torch.Tensor, g: Grid, gravity: float, vel: torch.Tensor, stream=None):
    _check(lib().awo_finalize(_dev(maxe, torch.float32, g.cells, "maxe"), g, gravity,
                              _dev(vel, torch.float32, g.cells, "vel"), _stream(stream)), "awo_finalize")


def lod_shapes(g: Grid, levels: int) -> list[tuple[int, int]]:
    """(height, width) of levels 0..levels-1."""
    out = [(int(g.height), int(g.width))]
    h, w = out[0]
    for _ in range(1, levels):
        h, w = (h + 1) // 2, (w + 1) // 2
        out.append((h, w))
    return out


def _lod_pointers(g: Grid, levels: int, count_lv: list, vel_lv: list):
    shapes = lod_shapes(g, levels)
    if len(count_lv) != levels - 1 or len(vel_lv) != levels - 1:
        raise ValueError("count_lv / vel_lv need levels-1 tensors")
    n = max(levels - 1, 1)
    cp = (ctypes.c_void_p * n)()
    vp = (ctypes.c_void_p * n)()
    for l in range(1, levels):
        hh, ww = shapes[l]
        cl, vl = count_lv[l - 1], vel_lv[l - 1]
        if cl.dtype not in (torch.int32, torch.uint32):
            raise TypeError("count_lv tensors must be int32 or uint32")
        cp[l - 1] = _dev(cl, cl.dtype, hh * ww, f"count_lv[{l - 1}]")
        vp[l - 1] = _dev(vl, torch.float32, hh * ww, f"vel_lv[{l - 1}]")
    return (cp, vp) if levels > 1 else (None, None)


def awo_overlay_lod(count: torch.Tensor, vel: torch.Tensor, g: Grid, levels: int, count_lv: list, vel_lv: list,
                    stream=None):
    cp, vp = _lod_pointers(g, levels, count_lv, vel_lv)
    _check(lib().awo_overlay_lod(_dev(count, count.dtype, g.cells, "count"), _dev(vel, torch.float32, g.cells, "vel"),
                                 g, int(levels), cp, vp, _stream(stream)), "awo_overlay_lod")


def awo_finalize_lod(maxe: torch.Tensor, count: torch.Tensor, g: Grid, gravity: float, levels: int,
                     vel: torch.Tensor, count_lv: list, vel_lv: list, stream=None):
    """awo_finalize then awo_overlay_lod in one pass (see awo.h)."""
    if count.dtype not in (torch.int32, torch.uint32):
        raise TypeError("count must be int32 or uint32")
    cp, vp = _lod_pointers(g, levels, count_lv, vel_lv)
    _check(lib().awo_finalize_lod(_dev(maxe, torch.float32, g.cells, "maxe"), _dev(count, count.dtype, g.cells, "count"),
                                  g, gravity, int(levels), _dev(vel, torch.float32, g.cells, "vel"), cp, vp,
                                  _stream(stream)), "awo_finalize_lod")


def awo_probe_threads() -> int:
    return int(lib().awo_probe_threads())


def awo_probe_l2_gather(buf: torch.Tensor, iters: int, sink: torch.Tensor, stream=None):
    _check(lib().awo_probe_l2_gather(_dev(buf, torch.int32, None, "buf"), buf.numel(), int(iters),
                                     _dev(sink, torch.int32, awo_probe_threads(), "sink"), _stream(stream)),
           "awo_probe_l2_gather")


def awo_probe_l2_red(buf: torch.Tensor, iters: int, stream=None):
    _check(lib().awo_probe_l2_red(_dev(buf, torch.int32, None, "buf"), buf.numel(), int(iters), _stream(stream)),
           "awo_probe_l2_red")


def awo_selftest_rcp_sqrt(first: int, count: int, out: torch.Tensor, stream=None):
    """Mismatches (into out, int64 [1] on the device) of the kernels' 1/sqrt against the IEEE intrinsics."""
    _check(lib().awo_selftest_rcp_sqrt(int(first), int(count), _dev(out, torch.int64, 1, "out"), _stream(stream)),
           "awo_selftest_rcp_sqrt")


def awo_selftest_visit_cell(first: int, count: int, out: torch.Tensor, stream=None):
    """Mismatches (into out, int64 [1] on the device) of the kernels' visited cell against nearest-centre."""
    _check(lib().awo_selftest_visit_cell(int(first), int(count), _dev(out, torch.int64, 1, "out"), _stream(stream)),
           "awo_selftest_visit_cell")


def awo_probe_philox(counters: torch.Tensor, seed: int, weyl_keys: bool, out: torch.Tensor, stream=None):
    """Philox4x32-10 words of the particle kernels for counters (int32 [n, 4]
    on the device, the words' bits) into out (int32 [n, 4]); round keys from
    the host table (weyl_keys False) or the Weyl schedule in registers."""
    if counters.dim() != 2 or counters.shape[1] != 4:
        raise ValueError("counters must be [n, 4]")
    n = counters.shape[0]
    _check(lib().awo_probe_philox(_dev(counters, torch.int32, None, "counters"), n, int(seed) & (2 ** 64 - 1),
                                  1 if weyl_keys else 0, _dev(out, torch.int32, 4 * n, "out"), _stream(stream)),
           "awo_probe_philox")


def awo_selftest_div_rn(divisors: torch.Tensor, span: int, out: torch.Tensor, stream=None):
    """Mismatches of the compose pass's refined division against the IEEE intrinsic, into out (int64 [1])."""
    _check(lib().awo_selftest_div_rn(_dev(divisors, torch.float32, None, "divisors"), int(divisors.numel()),
                                     int(span), _dev(out, torch.int64, 1, "out"), _stream(stream)),
           "awo_selftest_div_rn")


def awo_simulate_time_kernel(start, stop):
    """Hands two torch.cuda.Event objects (recorded once already, so that they
    exist) to the next awo_simulate of this thread, which records them around
    its particle kernel alone; None, None withdraws them."""
    if (start is None) != (stop is None):
        raise ValueError("give both events or neither")
    a = ctypes.c_void_p(start.cuda_event) if start is not None else None
    b = ctypes.c_void_p(stop.cuda_event) if stop is not None else None
    if start is not None and (not a.value or not b.value):
        raise ValueError("the events have not been created yet: record them once first")
    _check(lib().awo_simulate_time_kernel(a, b), "awo_simulate_time_kernel")


def stats_dict(stats: torch.Tensor) -> dict:
    """Host copy of an awo_sim_stats tensor (6 x int64 on the device)."""
    vals = stats.detach().to("cpu").tolist()
    return {k: int(v) & 0xFFFFFFFFFFFFFFFF for k, v in zip(STATS_FIELDS, vals)}


from .pipeline import Overlay  # noqa: E402  (re-export)
from .batch import Batch  # noqa: E402  (re-export)
from .differentiable import SoftDeposit, SoftOverlay  # noqa: E402  (re-export)
