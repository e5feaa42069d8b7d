"""Many regions through one batched particle launch, optionally as a CUDA graph.

``Batch`` holds one ``Overlay`` (device buffers) per region, runs the terrain
stages of every region, then ``awo_simulate_batched`` once for all regions,
then velocity and mipmap per region -- all on one stream.  ``capture()``
records that whole sequence in a CUDA graph (the library makes no host
synchronisation and no allocation, and the batched request table travels in
the kernel parameters), ``replay()`` relaunches it.  ``tune()`` runs the
library's autotuner on the batch.  Allocation and sequencing only; all
arithmetic runs in ``libawo.so``.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (SimParams, SimRequest, Tuning, awo_simulate_batched, awo_simulate_batched_workspace_bytes,
               awo_tune_batched, sim_request, stats_dict)
from .pipeline import SIM_CLEAR_OUTPUTS, Overlay, _ranged


def _per_region(x, n):
    return list(x) if isinstance(x, (list, tuple)) else [x] * n


class Batch:
    """Regions may differ in size, cell size, DEM storage (uint16 decimetres or
    float32 metres), mipmap depth and decode scale: pass a list for any of
    these, or one value for all."""

    def __init__(self, dems: list, cell_size, params: list[SimParams], release_deg: list[tuple[float, float]],
                 *, quantised, levels=1, decode_scale=0.1, device="cuda", load: bool = True):
        if not (len(dems) == len(params) == len(release_deg)):
            raise ValueError("dems, params and release ranges must have the same length")
        self.n = len(dems)
        self.decode_scale = _per_region(decode_scale, self.n)
        self.release_deg = list(release_deg)
        self.params = [SimParams.from_buffer_copy(p) for p in params]
        for p in self.params:
            p.flags |= SIM_CLEAR_OUTPUTS
        self.ovs = []
        for dem, cs, qz, lv, p in zip(dems, _per_region(cell_size, self.n), _per_region(quantised, self.n),
                                      _per_region(levels, self.n), self.params):
            H, W = dem.shape
            ov = Overlay(W, H, cs, quantised=qz, levels=lv, device=device, want_normals=False, want_mask=False,
                         release_log2=p.release_log2)
            if load:
                ov.load_dem(dem)
            self.ovs.append(ov)
        self.reqs = (SimRequest * self.n)()
        for i, ov in enumerate(self.ovs):
            self.reqs[i] = sim_request(ov.h, ov.g, ov.cells, ov.n_rel, ov.n_tex, self.params[i], ov.count,
                                       ov.maxe)
        self.ws = torch.empty(awo_simulate_batched_workspace_bytes(self.reqs) + 256, dtype=torch.uint8,
                              device=device)
        self.stats = torch.zeros((self.n, 6), dtype=torch.int64, device=device)
        self.tuning: Tuning | None = None
        self.graph: torch.cuda.CUDAGraph | None = None

    def terrain(self, stream=None):
        for ov, (lo, hi), sc in zip(self.ovs, self.release_deg, self.decode_scale):
            ov.terrain(lo, hi, sc, stream)

    @_ranged("awo simulate (batched)")
    def simulate(self, stream=None):
        awo_simulate_batched(self.reqs, self.ws, self.tuning, self.stats, stream)

    def overlay(self, stream=None):
        for ov, p in zip(self.ovs, self.params):
            ov.overlay(p.gravity, stream)

    def run(self, stream=None):
        self.terrain(stream)
        self.simulate(stream)
        self.overlay(stream)

    def tune(self) -> tuple[Tuning, float]:
        """Runs the terrain stages, then the library's autotuner on the batch."""
        self.terrain()
        best, ms = awo_tune_batched(self.reqs, self.ws)
        self.tuning = best
        return best, ms

    def capture(self) -> torch.cuda.CUDAGraph:
        self.run()  # warm caches (occupancy queries) outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()

    def stats_list(self) -> list[dict]:
        rows = self.stats.cpu().tolist()
        return [stats_dict(torch.tensor(r)) for r in rows]

    def results(self, i: int) -> dict:
        ov = self.ovs[i]
        return {"count": ov.count.cpu().numpy().view(np.uint32), "maxe": ov.maxe.cpu().numpy(),
                "vel": ov.vel.cpu().numpy(), "cells": ov.release_cells()}
