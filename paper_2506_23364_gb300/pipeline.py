"""The whole avalanche-overlay workflow on one GPU, through the C ABI.

``Overlay`` owns the device buffers of one DEM size and enqueues the calls of
the hot path on one CUDA stream: decode (for uint16 DEMs) -> normals ->
release -> simulate -> finalize -> mipmap.  The release count stays on the
device (``awo_simulate`` reads it), so a run needs no host synchronisation and
can be captured in a CUDA graph.  This module only allocates and sequences;
all arithmetic runs in ``libawo.so``.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (AWO_OK, Grid, SimParams, awo_finalize_lod, awo_normals, awo_normals_u16,
               awo_release, awo_release_from_mask, awo_release_texture, awo_release_texture_dims,
               awo_release_texture_workspace_bytes, awo_release_workspace_bytes, awo_simulate,
               awo_simulate_workspace_bytes, grid, lod_shapes, stats_dict)

SIM_CLEAR_OUTPUTS = 1


def _ranged(name: str):
    """Wraps a stage in an NVTX range (visible in a profiler's timeline)."""
    def deco(fn):
        def wrapped(*args, **kwargs):
            torch.cuda.nvtx.range_push(name)
            try:
                return fn(*args, **kwargs)
            finally:
                torch.cuda.nvtx.range_pop()
        wrapped.__doc__ = fn.__doc__
        wrapped.__name__ = fn.__name__
        return wrapped
    return deco


def _ws(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 16) + 256, dtype=torch.uint8, device=device)


class Overlay:
    """Device buffers and call sequence for one W x H workflow.

    ``release_log2`` = r evaluates release points on a texture at 2^r times
    the DEM's resolution (r in -3..3; 0: one per cell): the mask and the
    release list are then at that texture's resolution, and the particles
    start at texel centres."""

    def __init__(self, width: int, height: int, cell_size: float, *, quantised: bool, levels: int = 1,
                 device="cuda", want_normals: bool = True, want_slope: bool = False, want_mask: bool = True,
                 release_log2: int = 0):
        self.g: Grid = grid(width, height, cell_size)
        self.levels = int(levels)
        self.quantised = quantised
        self.release_log2 = int(release_log2)
        d = torch.device(device)
        self.device = d
        if self.release_log2:
            wr, hr = awo_release_texture_dims(self.g, self.release_log2)
            self.g_rel: Grid = grid(wr, hr, cell_size * 2.0 ** (-self.release_log2))
        else:
            self.g_rel = self.g
        n_rel = self.g_rel.cells
        self.n_tex = n_rel
        self.q = torch.empty((height, width), dtype=torch.int16, device=d) if quantised else None
        self.h = torch.empty((height, width), dtype=torch.float32, device=d)
        self.normal = torch.empty((3, height, width), dtype=torch.float32, device=d) if want_normals else None
        self.tan2 = torch.empty((height, width), dtype=torch.float32, device=d)
        self.slope = torch.empty((height, width), dtype=torch.float32, device=d) if want_slope else None
        want_mask = want_mask or bool(self.release_log2)  # the texture path needs its mask
        self.mask = torch.empty((self.g_rel.height, self.g_rel.width), dtype=torch.uint8, device=d) \
            if want_mask else None
        self.cells = torch.empty(n_rel, dtype=torch.int32, device=d)
        self.n_rel = torch.zeros(1, dtype=torch.int32, device=d)
        self.ws_rel = _ws(awo_release_texture_workspace_bytes(self.g, self.release_log2) if self.release_log2
                          else awo_release_workspace_bytes(self.g), d)
        self.ws_sim = _ws(awo_simulate_workspace_bytes(n_rel), d)
        self.count = torch.zeros((height, width), dtype=torch.int32, device=d)
        self.maxe = torch.zeros((height, width), dtype=torch.float32, device=d)
        self.vel = torch.empty((height, width), dtype=torch.float32, device=d)
        self.stats = torch.zeros(6, dtype=torch.int64, device=d)
        shapes = lod_shapes(self.g, self.levels)
        self.count_lv = [torch.empty(s, dtype=torch.int32, device=d) for s in shapes[1:]]
        self.vel_lv = [torch.empty(s, dtype=torch.float32, device=d) for s in shapes[1:]]

    # ------------------------------------------------------------------
    def load_dem(self, dem: np.ndarray | torch.Tensor, non_blocking: bool = False):
        """Copies a host DEM (uint16 decimetres or float32 metres) to the device."""
        if self.quantised:
            src = torch.from_numpy(np.ascontiguousarray(dem).view(np.int16)) if isinstance(dem, np.ndarray) else dem
            self.q.copy_(src.view(torch.int16) if src.dtype != torch.int16 else src, non_blocking=non_blocking)
        else:
            src = torch.from_numpy(np.ascontiguousarray(dem, dtype=np.float32)) if isinstance(dem, np.ndarray) else dem
            self.h.copy_(src, non_blocking=non_blocking)

    @_ranged("awo terrain")
    def terrain(self, slope_lo_deg: float, slope_hi_deg: float, decode_scale: float = 0.1, stream=None):
        """a0-b: decode, normals and release (the count stays on the device)."""
        if self.quantised:  # decode and normals in one pass
            awo_normals_u16(self.q, self.g, decode_scale, self.h, self.normal, self.tan2, self.slope, stream)
        else:
            awo_normals(self.h, self.g, self.normal, self.tan2, self.slope, stream)
        if self.release_log2:
            awo_release_texture(self.tan2, self.g, self.release_log2, slope_lo_deg, slope_hi_deg, self.mask,
                                self.cells, self.n_rel, self.ws_rel, stream)
        else:
            awo_release(self.tan2, self.g, slope_lo_deg, slope_hi_deg, self.mask, self.cells, self.n_rel,
                        self.ws_rel, stream)

    @_ranged("awo terrain (mask)")
    def terrain_from_mask(self, mask: torch.Tensor, decode_scale: float = 0.1, stream=None):
        """a0-b': decode, normals and the release list from a caller's uint8
        mask (at the release texture's resolution)."""
        if self.quantised:
            awo_normals_u16(self.q, self.g, decode_scale, self.h, self.normal, self.tan2, self.slope, stream)
        else:
            awo_normals(self.h, self.g, self.normal, self.tan2, self.slope, stream)
        awo_release_from_mask(mask, self.g_rel, self.cells, self.n_rel, self.ws_rel, stream)

    @_ranged("awo simulate")
    def simulate(self, params: SimParams, clear: bool = True, stream=None, cells=None, n_cells=None):
        """c: particles from the release list (or from the given cells)."""
        p = SimParams.from_buffer_copy(params)
        p.release_log2 = self.release_log2
        if clear:
            p.flags |= SIM_CLEAR_OUTPUTS
        if cells is None:
            awo_simulate(self.h, self.g, self.cells, self.n_rel, self.n_tex, p, self.count, self.maxe, self.stats,
                         self.ws_sim, stream)
        else:
            awo_simulate(self.h, self.g, cells, None, int(n_cells), p, self.count, self.maxe, self.stats,
                         self.ws_sim, stream)

    @_ranged("awo overlay")
    def overlay(self, gravity: float = 9.81, stream=None):
        """c'-d: velocity indicator and mipmap, in one pass."""
        awo_finalize_lod(self.maxe, self.count, self.g, gravity, self.levels, self.vel, self.count_lv, self.vel_lv,
                         stream)

    def run(self, slope_lo_deg: float, slope_hi_deg: float, params: SimParams, decode_scale: float = 0.1,
            stream=None):
        self.terrain(slope_lo_deg, slope_hi_deg, decode_scale, stream)
        self.simulate(params, True, stream)
        self.overlay(params.gravity, stream)

    def capture(self, slope_lo_deg: float, slope_hi_deg: float, params: SimParams,
                decode_scale: float = 0.1) -> torch.cuda.CUDAGraph:
        """Records the whole workflow (from the DEM already on the device) in a
        CUDA graph; ``replay()`` relaunches it after the DEM buffer is refilled,
        with no per-kernel host work.  The library makes no host
        synchronisation and no allocation inside the calls, and the release
        count stays on the device, so the graph is the same for every DEM."""
        self.run(slope_lo_deg, slope_hi_deg, params, decode_scale)  # warm per-device caches outside the capture
        torch.cuda.synchronize(self.device)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.run(slope_lo_deg, slope_hi_deg, params, decode_scale)
        self.graph = graph
        return graph

    def replay(self):
        if getattr(self, "graph", None) is None:
            raise RuntimeError("capture() first")
        self.graph.replay()

    # ------------------------------------------------------------------
    def n_release(self) -> int:
        return int(self.n_rel.item())

    def release_cells(self) -> np.ndarray:
        k = self.n_release()
        return self.cells[:k].cpu().numpy().view(np.uint32)

    def stats_dict(self) -> dict:
        return stats_dict(self.stats)

    def host_results(self) -> dict:
        out = {"tan2": self.tan2.cpu().numpy(), "count": self.count.cpu().numpy().view(np.uint32),
               "maxe": self.maxe.cpu().numpy(), "vel": self.vel.cpu().numpy(),
               "cells": self.release_cells(), "stats": self.stats_dict(),
               "count_lv": [self.count.cpu().numpy().view(np.uint32)] + [c.cpu().numpy().view(np.uint32)
                                                                        for c in self.count_lv],
               "vel_lv": [self.vel.cpu().numpy()] + [v.cpu().numpy() for v in self.vel_lv]}
        if self.normal is not None:
            out["normals"] = self.normal.cpu().numpy()
        if self.slope is not None:
            out["slope_deg"] = self.slope.cpu().numpy()
        if self.mask is not None:
            out["mask"] = self.mask.cpu().numpy()
        if self.quantised:
            out["h"] = self.h.cpu().numpy()
        return out
