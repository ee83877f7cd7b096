"""Differentiable march: a torch.autograd.Function over rt_advance / rt_backward.

The forward pass is one rt_advance; the backward pass is the hand-written reverse-march
adjoint (rt_backward / rt_backward_sources), which recomputes the forward state from per-ray
checkpoints. Gradients flow to j and kappa (the Jacobians w.r.t. (j, kappa) of Sec. 4) and,
when the source tensor requires it, to the source positions; the step length, c and dt are
not differentiated. Parameters that build j or kappa (a global kappa scale, per-source
amplitudes, per-bin factors) get their gradients from torch's chain rule through these.
"""
from __future__ import annotations

import torch

from .api import Grid, _cached_grid, _grid_tensor


class RTFunction(torch.autograd.Function):
    """field = RTFunction.apply(j, kappa, sources, num_rays, step_size, radiation_velocity,
    time_step, grid); j, kappa: [n_freq, n0, n1, n2] CUDA float32 (or 3-D for one bin)."""

    @staticmethod
    def forward(ctx, j, kappa, sources, num_rays, step_size, radiation_velocity, time_step, grid):
        squeeze = j.dim() == 3
        j4 = _grid_tensor(j, "j")
        k4 = _grid_tensor(kappa, "kappa")
        if grid is None:
            # the forward records the reverse march's checkpoints; backward reuses them
            grid = _cached_grid(j4.shape[1:], j4.shape[0], j4.device, record_checkpoints=True)
        # one device copy of the sources, used by both passes (the recorded checkpoints are
        # matched by buffer address)
        src = torch.as_tensor(sources, dtype=torch.float32, device=j4.device).detach().reshape(-1, 3).contiguous()
        out = grid.advance(j4, k4, src, num_rays, step_size, radiation_velocity, time_step)
        ctx.save_for_backward(j4, k4, src)
        ctx.src_shape = tuple(torch.as_tensor(sources).shape)
        ctx.args = (num_rays, step_size, radiation_velocity, time_step, grid, squeeze)
        return out[0] if squeeze else out

    @staticmethod
    def backward(ctx, grad_out):
        j4, k4, src = ctx.saved_tensors
        num_rays, step_size, c, dt, grid, squeeze = ctx.args
        g = grad_out.unsqueeze(0) if squeeze else grad_out
        need_j, need_k, need_s = ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2]
        res = grid.backward(g.contiguous().float(), j4, k4, src, num_rays, step_size, c, dt,
                            need_j=need_j, need_kappa=need_k, need_sources=need_s)
        gj, gk = res[0], res[1]
        gs = res[2].reshape(ctx.src_shape) if need_s else None
        if squeeze:
            gj = gj[0] if gj is not None else None
            gk = gk[0] if gk is not None else None
        return gj, gk, gs, None, None, None, None, None


def render(j, kappa, sources, num_rays: int, step_size: float, radiation_velocity: float = 1.0,
           time_step: float = 1.0, grid: Grid | None = None) -> torch.Tensor:
    """Differentiable one-dt field (see RTFunction)."""
    return RTFunction.apply(j, kappa, sources, num_rays, step_size, radiation_velocity, time_step, grid)
