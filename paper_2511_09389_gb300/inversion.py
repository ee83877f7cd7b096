"""Gradient-based recovery of the emissivity from a target field (Sec. 4, "Gradient-based
inversion", generalised from the paper's single amplitude to every voxel of j).

The loss is the mean squared difference of log fields,
    L(j) = mean_v (log(F(j)_v + eps) - log(F_target_v + eps))^2,   eps = eps_rel * max F_target,
(the field vanishes past the light-travel horizon, so eps keeps the logarithm finite). F(j) is
one rt_advance through RTFunction, dL/dj the hand-written reverse march. j starts from zero and
takes Adam steps (the library's rt_adam_step kernel), each followed by a projection onto j >= 0:
a negative emissivity would make the field negative where the logarithm is undefined.

The floor eps defaults to 1e-2 of the target's maximum. At j = 0 the field is zero and the
gradient of the loss scales as 1/eps; with a floor of 1e-8 of the maximum that first gradient
(~1e6) fills Adam's second moment, which forgets it only over ~1/(1 - beta2) = 1000 steps, so
every later step is a tiny fraction of the learning rate (measured with the FP64 oracle on 16^3:
the peak of j reached 0.06 of 4.5 in 100 steps, correlation with the true j 0.03). With a floor
of 1e-2 the same run recovers the blobs (correlation 0.65); the field below 1 % of its peak,
far from every blob, then weighs less in the loss.
"""
from __future__ import annotations

import time

import torch

from .api import Grid, adam_step
from .autograd import RTFunction


def log_field_loss(F: torch.Tensor, log_target: torch.Tensor, eps: float) -> torch.Tensor:
    """mean((log(F + eps) - log_target)^2), differentiable in F."""
    return ((torch.log(F + eps) - log_target) ** 2).mean()


def recover_emissivity(target: torch.Tensor, kappa: torch.Tensor, sources: torch.Tensor, num_rays: int,
                       step_size: float, radiation_velocity: float, time_step: float, *, iterations: int = 200,
                       lr: float = 1e-2, eps_rel: float = 1e-2, grid: Grid | None = None, j0=None) -> dict:
    """Recover j (same shape as kappa) whose field matches `target` (the field of the unknown
    emissivity, same shape) in the log-MSE sense. Returns the recovered j, the loss before every
    step and after the last, and the wall time of the iterations (synchronised at the end)."""
    dev = kappa.device
    if grid is None:
        shape = tuple(kappa.shape[-3:])
        nf = 1 if kappa.dim() == 3 else kappa.shape[0]
        grid = Grid(shape, nf, record_checkpoints=True, autotune=True, device=dev)
    eps = eps_rel * float(target.max())
    log_t = torch.log(target + eps)
    j = torch.zeros_like(kappa) if j0 is None else j0.detach().clone().float()
    m, v = torch.zeros_like(j), torch.zeros_like(j)
    losses = []
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for it in range(1, iterations + 1):
        jv = j.detach().requires_grad_(True)
        F = RTFunction.apply(jv, kappa, sources, num_rays, step_size, radiation_velocity, time_step, grid)
        loss = log_field_loss(F, log_t, eps)
        loss.backward()
        losses.append(loss.detach())
        adam_step(j, jv.grad, m, v, lr=lr, step=it)
        j.clamp_(min=0.0)
    with torch.no_grad():
        F = RTFunction.apply(j, kappa, sources, num_rays, step_size, radiation_velocity, time_step, grid)
        losses.append(log_field_loss(F, log_t, eps))
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    return {"j": j, "losses": [float(x) for x in torch.stack(losses).cpu()], "wall_s": wall,
            "iterations": iterations, "ckpt_stride": grid.last_ckpt_stride()}


def correlation(a: torch.Tensor, b: torch.Tensor) -> float:
    """Pearson correlation of two fields over all voxels."""
    x = a.double().flatten() - a.double().mean()
    y = b.double().flatten() - b.double().mean()
    return float((x @ y) / (x.norm() * y.norm()))
