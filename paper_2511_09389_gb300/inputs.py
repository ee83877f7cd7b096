"""Seeded synthetic inputs for the march (shared by the oracle tests and the CUDA path).

This module only makes inputs: it holds none of the method's arithmetic (no ray geometry,
no interpolation, no transport update). Both the FP64 oracle and the CUDA library receive
the same arrays from here.

The paper's turbulent media are hydro snapshots (Sec. 3, "Turbulent snapshots from hydro")
that are not available; a seeded lognormal field with a Kolmogorov-like spectrum stands in:
white noise N(0, 1) on the periodic N^3 grid (numpy PCG64) -> FFT -> times sqrt(P(k)) with
P(k) ~ |k|^(-11/3), P(0) = 0 -> inverse FFT -> g / std(g) * sigma_g -> kappa = exp(g),
rescaled to the requested mean per cell. Emissivity j is a sum of isotropic Gaussian blobs
evaluated at integer voxel coordinates; sources sit at the blob centres or at seeded
positions. All arrays are float32, C-contiguous, axis order [bin][axis0][axis1][axis2].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def lognormal_field(shape, sigma_g: float, mean: float, seed: int) -> np.ndarray:
    """exp of a Gaussian random field with P(k) ~ k^(-11/3), rescaled to the given mean."""
    shape = tuple(int(s) for s in shape)
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.standard_normal(shape)
    fk = np.fft.rfftn(noise)
    kx = np.fft.fftfreq(shape[0])[:, None, None]
    ky = np.fft.fftfreq(shape[1])[None, :, None]
    kz = np.fft.rfftfreq(shape[2])[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (-11.0 / 12.0)          # sqrt(P), P ~ |k|^(-11/3)
    g = np.fft.irfftn(fk * amp, s=shape, axes=(0, 1, 2))
    g = g / g.std() * sigma_g
    kap = np.exp(g)
    kap *= mean / kap.mean()
    return kap.astype(np.float32)


def gaussian_blobs(shape, centres, sigmas, amplitudes) -> np.ndarray:
    """j[v] = sum_i A_i exp(-|v - c_i|^2 / (2 sigma_i^2)) at integer voxel coordinates v."""
    shape = tuple(int(s) for s in shape)
    out = np.zeros(shape, np.float64)
    ax = [np.arange(n, dtype=np.float64) for n in shape]
    for c, s, a in zip(np.atleast_2d(centres), np.broadcast_to(sigmas, (len(np.atleast_2d(centres)),)),
                       np.broadcast_to(amplitudes, (len(np.atleast_2d(centres)),))):
        g0 = np.exp(-(ax[0] - c[0]) ** 2 / (2 * s * s))
        g1 = np.exp(-(ax[1] - c[1]) ** 2 / (2 * s * s))
        g2 = np.exp(-(ax[2] - c[2]) ** 2 / (2 * s * s))
        out += a * g0[:, None, None] * g1[None, :, None] * g2[None, None, :]
    return out.astype(np.float32)


@dataclass
class Problem:
    """One march problem: inputs plus the scalar arguments of an advance call."""
    name: str
    j: np.ndarray                 # [n_freq, n0, n1, n2] float32
    kappa: np.ndarray             # [n_freq, n0, n1, n2] float32
    sources: np.ndarray           # [n_src, 3] float32, grid coordinates
    num_rays: int
    step_size: float
    radiation_velocity: float
    time_step: float
    extra: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.j.shape[1:]

    @property
    def n_freq(self):
        return self.j.shape[0]


def single_source_uniform(n: int = 32, kappa0: float = 0.1, sigma: float = 1.0, amp: float = 1.0,
                          num_rays: int = 768, step_size: float = 0.5, horizon: float = 16.0) -> Problem:
    """Plain single-source march: uniform kappa, one Gaussian blob and one source at the grid
    centre ((n-1)/2 per axis), one bin. Defaults: 32^3, kappa 0.1, N_Omega 768, ds 0.5,
    c dt 16 (N_s = 32)."""
    c = np.full(3, (n - 1) / 2.0)
    j = gaussian_blobs((n, n, n), c[None], sigma, amp)[None]
    kap = np.full((1, n, n, n), kappa0, np.float32)
    return Problem("single_source_uniform", j, kap, c[None].astype(np.float32), num_rays,
                   step_size, 1.0, horizon)


def turbulent(n: int = 128, n_src: int = 16, num_rays: int = 3072, step_size: float = 0.5,
              horizon: float = 128.0, nu_ratios=(1.0, 1.3, 1.8, 2.5), sigma_g: float = 1.0,
              kappa_mean: float = 0.05, blob_sigma: float = 1.5, seed: int = 2000) -> Problem:
    """Turbulent medium: lognormal kappa (sigma_g 1, mean 0.05), n_src sources uniform in
    [0, n-1]^3 with Gaussian blobs (sigma 1.5, amplitude log-uniform in [0.1, 10]), bins with
    kappa scaled by (nu/nu0)^-3 and the same j. Defaults: 128^3, 16 sources, N_Omega 3072,
    ds 0.5, c dt 128 (N_s 256), 4 bins."""
    kap0 = lognormal_field((n, n, n), sigma_g, kappa_mean, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    src = rng.uniform(0.0, n - 1.0, size=(n_src, 3))
    amps = 10.0 ** rng.uniform(-1.0, 1.0, size=n_src)
    j0 = gaussian_blobs((n, n, n), src, blob_sigma, amps)
    nf = len(nu_ratios)
    j = np.broadcast_to(j0, (nf, n, n, n)).copy()
    kap = np.stack([(kap0.astype(np.float64) * r ** -3.0).astype(np.float32) for r in nu_ratios])
    return Problem("turbulent", j, kap, src.astype(np.float32), num_rays, step_size, 1.0, horizon,
                   extra={"seed": seed, "nu_ratios": tuple(nu_ratios)})


def paper_timing(n: int = 128, fraction: float = 0.001, num_rays: int = 4096, step_size: float = 0.5,
                 horizon: float = 128.0, blob_sigma: float = 1.5, seed: int = 5000) -> Problem:
    """The paper's timing run (Sec. 2; sources placed as in Sec. 3) with a synthetic medium:
    lognormal kappa on 128^3 (sigma_g 1, mean 0.05), sources at the `fraction` = 0.1 % cells of
    highest kappa (2097), each the centre of a Gaussian j blob (sigma 1.5, amplitude log-uniform
    in [0.1, 10]), N_Omega 4096, ds 0.5, one bin. The paper does not state its horizon; c dt =
    128 (N_s 256) is assumed. Sources are listed by decreasing kappa (ties by cell index)."""
    kap = lognormal_field((n, n, n), 1.0, 0.05, seed)
    n_src = int(round(fraction * n ** 3))
    flat = kap.reshape(-1).astype(np.float64)
    order = np.lexsort((np.arange(flat.size), -flat))[:n_src]
    src = np.stack(np.unravel_index(order, (n, n, n)), axis=1).astype(np.float64)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    amps = 10.0 ** rng.uniform(-1.0, 1.0, size=n_src)
    # j = sum_i A_i g(x - c_i0) g(y - c_i1) g(z - c_i2): a sum of separable terms, as contractions
    ax = np.arange(n, dtype=np.float64)
    g = [np.exp(-(ax[None, :] - src[:, a, None]) ** 2 / (2 * blob_sigma ** 2)) for a in range(3)]
    j = np.empty((n, n, n))
    for x in range(n):
        j[x] = (g[1] * (amps * g[0][:, x])[:, None]).T @ g[2]
    return Problem("paper_timing", j.astype(np.float32)[None], kap[None], src.astype(np.float32), num_rays,
                   step_size, 1.0, horizon, extra={"seed": seed, "fraction": fraction})


def inverse_problem(n: int = 64, n_blobs: int = 8, num_rays: int = 3072, step_size: float = 0.5,
                    horizon: float = 64.0, seed: int = 4000) -> Problem:
    """Differentiable inverse problem: lognormal kappa (sigma_g 1, mean 0.05); target j made of
    n_blobs Gaussian blobs (sigma 2, seeded positions and amplitudes); sources at the blob
    centres. Defaults: 64^3, 8 blobs, N_Omega 3072, ds 0.5, N_s 128."""
    kap = lognormal_field((n, n, n), 1.0, 0.05, seed)[None]
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    c = rng.uniform(4.0, n - 5.0, size=(n_blobs, 3))
    amps = 10.0 ** rng.uniform(-0.5, 0.5, size=n_blobs)
    j = gaussian_blobs((n, n, n), c, 2.0, amps)[None]
    return Problem("inverse_problem", j, kap, c.astype(np.float32), num_rays, step_size, 1.0,
                   horizon, extra={"seed": seed})


def batch_instances(count: int = 64, seed: int = 3000, edges=(32, 48, 64, 96, 128, 160),
                    ray_choices=(768, 3072, 12288), max_src: int = 64, max_freq: int = 8):
    """Batched workload: independent instances with edge from `edges`, sigma_g in [0.5, 1.5],
    1..max_src sources, N_Omega from `ray_choices`, ds 0.5, c dt = edge, 1..max_freq bins with
    kappa scaled by (nu/nu0)^-3 over nu/nu0 evenly spaced in [1, 2.5]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(rng.choice(edges))
        sg = float(rng.uniform(0.5, 1.5))
        ns = int(rng.integers(1, max_src + 1))
        nr = int(rng.choice(ray_choices))
        nf = int(rng.integers(1, max_freq + 1))
        kap0 = lognormal_field((n, n, n), sg, 0.05, seed * 100 + i)
        src = rng.uniform(0.0, n - 1.0, size=(ns, 3))
        amps = 10.0 ** rng.uniform(-1.0, 1.0, size=ns)
        j0 = gaussian_blobs((n, n, n), src, 1.5, amps)
        ratios = np.linspace(1.0, 2.5, nf) if nf > 1 else np.ones(1)
        j = np.broadcast_to(j0, (nf, n, n, n)).copy()
        kap = np.stack([(kap0.astype(np.float64) * r ** -3.0).astype(np.float32) for r in ratios])
        out.append(Problem(f"instance{i}", j, kap, src.astype(np.float32), nr, 0.5, 1.0, float(n),
                           extra={"sigma_g": sg}))
    return out


def surrogate_sample(seed: int, n: int = 64, num_rays: int = 3072, step_size: float = 0.5,
                     horizon: float = 64.0) -> Problem:
    """One surrogate training/held-out pair input: lognormal kappa with sigma_g in [0.5, 1.5],
    1..8 Gaussian sources (sigma 1.5, amplitude log-uniform in [0.1, 10]), one bin."""
    rng = np.random.Generator(np.random.PCG64(5_000_000 + seed))
    sg = float(rng.uniform(0.5, 1.5))
    ns = int(rng.integers(1, 9))
    kap = lognormal_field((n, n, n), sg, 0.05, 5_100_000 + seed)[None]
    src = rng.uniform(4.0, n - 5.0, size=(ns, 3))
    amps = 10.0 ** rng.uniform(-1.0, 1.0, size=ns)
    j = gaussian_blobs((n, n, n), src, 1.5, amps)[None]
    return Problem(f"surrogate{seed}", j, kap, src.astype(np.float32), num_rays, step_size, 1.0,
                   horizon, extra={"sigma_g": sg})


def random_small(seed: int, shape=(9, 7, 11), n_freq: int = 2, n_src: int = 3, num_rays: int = 37,
                 step_size: float = 0.75, horizon: float = 9.0, outside: bool = True) -> Problem:
    """Small irregular problem for parity tests: non-cubic grid, random positive kappa and j,
    some sources near or outside the faces so rays leave the box (clamped deposits)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = tuple(shape)
    j = rng.uniform(0.0, 1.0, size=(n_freq,) + shape).astype(np.float32)
    kap = rng.uniform(0.0, 0.4, size=(n_freq,) + shape).astype(np.float32)
    lo = -1.5 if outside else 0.0
    src = np.stack([rng.uniform(lo, s - 1 - lo, size=n_src) for s in shape], axis=1)
    return Problem(f"random_small{seed}", j, kap, src.astype(np.float32), num_rays, step_size, 1.0,
                   horizon)


def surrogate_batch_torch(seeds, n: int = 64, device="cuda"):
    """Surrogate training / held-out inputs generated on the GPU (torch), one per seed: the
    same recipe as surrogate_sample (lognormal kappa with sigma_g in [0.5, 1.5] and mean 0.05,
    1..8 Gaussian sources of sigma 1.5 with amplitude log-uniform in [0.1, 10], placed in
    [4, n-5]^3), drawn from torch generators seeded per sample. Returns kappa [B, n, n, n],
    j [B, n, n, n] (float32, on `device`) and a list of [n_src, 3] float32 source tensors."""
    import torch
    B = len(seeds)
    kap = torch.empty((B, n, n, n), dtype=torch.float32, device=device)
    jj = torch.zeros((B, n, n, n), dtype=torch.float32, device=device)
    f = torch.fft.fftfreq(n, device=device, dtype=torch.float64)
    fr = torch.fft.rfftfreq(n, device=device, dtype=torch.float64)
    k2 = f[:, None, None] ** 2 + f[None, :, None] ** 2 + fr[None, None, :] ** 2
    amp = torch.where(k2 > 0, k2.clamp_min(1e-30) ** (-11.0 / 12.0), torch.zeros_like(k2))
    ax = torch.arange(n, device=device, dtype=torch.float32)
    sources = []
    for b, s in enumerate(seeds):
        g = torch.Generator(device=device)
        g.manual_seed(7_000_000 + int(s))
        h = torch.Generator(device="cpu")
        h.manual_seed(8_000_000 + int(s))
        sg = 0.5 + torch.rand((), generator=h).item()
        ns = int(torch.randint(1, 9, (), generator=h).item())
        noise = torch.randn((n, n, n), generator=g, device=device, dtype=torch.float64)
        gr = torch.fft.irfftn(torch.fft.rfftn(noise) * amp, s=(n, n, n))
        gr = gr / gr.std() * sg
        kk = torch.exp(gr)
        kap[b] = (kk * (0.05 / kk.mean())).float()
        src = 4.0 + torch.rand((ns, 3), generator=h) * (n - 9.0)
        amps = 10.0 ** (torch.rand(ns, generator=h) * 2.0 - 1.0)
        for c, a in zip(src.to(device), amps.to(device)):
            g0 = torch.exp(-(ax - c[0]) ** 2 / 4.5)
            g1 = torch.exp(-(ax - c[1]) ** 2 / 4.5)
            g2 = torch.exp(-(ax - c[2]) ** 2 / 4.5)
            jj[b] += a * g0[:, None, None] * g1[None, :, None] * g2[None, None, :]
        sources.append(src.float().to(device))
    return kap, jj, sources
