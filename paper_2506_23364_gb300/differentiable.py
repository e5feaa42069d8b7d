"""Differentiable soft-deposit overlay: friction parameters and release
weights fitted by gradient descent through the library's adjoint kernel.

``SoftOverlay`` prepares one DEM (terrain stages and the release list run
once through the library) and exposes ``deposit(log_mu, log_k, weights)``,
the soft-deposit raster D as a differentiable torch function:
``SoftDeposit.forward`` runs ``awo_soft_forward`` and ``SoftDeposit.backward``
runs ``awo_soft_backward`` (exact vector-Jacobian product; parameters enter
through log(mu) and log(drag_k)).  Marshalling only; all arithmetic runs in
``libawo.so``.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import (SimParams, awo_fixed_to_real, awo_soft_backward, awo_soft_forward, awo_soft_workspace_bytes)
from .pipeline import SIM_CLEAR_OUTPUTS, Overlay


class SoftOverlay:
    def __init__(self, dem: np.ndarray, cell_size: float, release_deg: tuple[float, float], *,
                 traj_per_cell: int, max_steps: int, persistence: float = 0.9, randomness: float = 0.16,
                 step_scale: float = 1.0, seed: int = 0, tau: float = 1.0, decode_scale: float = 0.1,
                 device="cuda"):
        H, W = dem.shape
        self.ov = Overlay(W, H, cell_size, quantised=dem.dtype == np.uint16, levels=1, device=device,
                          want_normals=False, want_mask=False)
        self.ov.load_dem(dem)
        self.ov.terrain(*release_deg, decode_scale)
        self.n_cells = self.ov.n_release()
        self.cells = self.ov.cells[: max(self.n_cells, 1)]
        self.base = dict(persistence=persistence, randomness=randomness, step_scale=step_scale,
                         traj_per_cell=traj_per_cell, max_steps=max_steps, seed=seed)
        self.tau = float(tau)
        self.g = self.ov.g
        self.device = self.ov.device
        self.ws = torch.empty(awo_soft_workspace_bytes(self.n_cells) + 256, dtype=torch.uint8, device=device)
        self.q = torch.zeros((H, W), dtype=torch.int64, device=device)
        self.stats = torch.zeros(6, dtype=torch.int64, device=device)

    def params(self, mu: float, drag_k: float, clear: bool = True) -> SimParams:
        p = SimParams.make(mu=mu, drag_k=drag_k, **self.base)
        if clear:
            p.flags |= SIM_CLEAR_OUTPUTS
        return p

    def forward_raw(self, mu: float, drag_k: float, weights: torch.Tensor) -> torch.Tensor:
        """D (FP64 [H, W]) at fixed parameters, no autograd."""
        awo_soft_forward(self.ov.h, self.g, self.cells, None, self.n_cells, weights, self.params(mu, drag_k),
                         self.tau, self.q, self.stats, self.ws)
        D = torch.empty(self.q.shape, dtype=torch.float64, device=self.device)
        awo_fixed_to_real(self.q, D)
        return D

    def backward_raw(self, mu: float, drag_k: float, weights: torch.Tensor, G: torch.Tensor):
        """(dL/dlog mu, dL/dlog k) FP64 [2] and dL/dw FP32 [n_cells] for G = dL/dD."""
        gt = torch.empty(2, dtype=torch.float64, device=self.device)
        gw = torch.empty(max(self.n_cells, 1), dtype=torch.float32, device=self.device)
        awo_soft_backward(self.ov.h, self.g, self.cells, None, self.n_cells, weights, self.params(mu, drag_k),
                          self.tau, G.to(torch.float32).contiguous(), gt, gw, self.ws)
        return gt, gw[: self.n_cells]

    def deposit(self, log_mu: torch.Tensor, log_k: torch.Tensor, weights: torch.Tensor) -> torch.Tensor:
        return SoftDeposit.apply(log_mu, log_k, weights, self)


class SoftDeposit(torch.autograd.Function):
    """D(log mu, log k, w): forward and exact backward through the library."""

    @staticmethod
    def forward(ctx, log_mu, log_k, weights, prob: SoftOverlay):
        mu, k = math.exp(float(log_mu)), math.exp(float(log_k))
        w = weights.detach().to(device=prob.device, dtype=torch.float32).contiguous()
        D = prob.forward_raw(mu, k, w)
        ctx.prob, ctx.mu, ctx.k = prob, mu, k
        ctx.save_for_backward(w)
        ctx.meta = tuple((torch.as_tensor(t).shape, torch.as_tensor(t).dtype, torch.as_tensor(t).device)
                         for t in (log_mu, log_k))
        return D

    @staticmethod
    def backward(ctx, gD):
        (w,) = ctx.saved_tensors
        gt, gw = ctx.prob.backward_raw(ctx.mu, ctx.k, w, gD)
        (sm, dm, vm), (sk, dk, vk) = ctx.meta
        g_mu = gt[0].to(device=vm, dtype=dm).reshape(sm)
        g_k = gt[1].to(device=vk, dtype=dk).reshape(sk)
        return g_mu, g_k, gw.to(torch.float32), None
