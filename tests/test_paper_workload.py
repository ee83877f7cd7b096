"""The paper's timing workload generator (sources at the highest-kappa cells, Gaussian j
blobs), checked on a small grid against its definition; the GPU march on the full-size
workload against the oracle (a source subset) and against the sum over sources of separate runs."""
import os

import numpy as np
import pytest

import oracle
from paper_2511_09389_gb300 import inputs


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2511_09389_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


def test_generator_small():
    p = inputs.paper_timing(n=24, fraction=0.01, num_rays=64)
    n_src = int(round(0.01 * 24 ** 3))
    assert p.sources.shape == (n_src, 3) and p.n_freq == 1 and p.num_rays == 64
    k = p.kappa[0].astype(np.float64)
    idx = p.sources.astype(np.int64)
    assert np.array_equal(idx.astype(np.float32), p.sources)       # cell centres, integer coordinates
    ks = k[idx[:, 0], idx[:, 1], idx[:, 2]]
    rest = np.ones(k.shape, bool)
    rest[idx[:, 0], idx[:, 1], idx[:, 2]] = False
    assert len({tuple(r) for r in idx}) == n_src
    assert ks.min() >= k[rest].max() and np.all(np.diff(ks) <= 0)  # the top cells, by decreasing kappa
    rng = np.random.Generator(np.random.PCG64(5001))
    amps = 10.0 ** rng.uniform(-1.0, 1.0, size=n_src)
    ref = inputs.gaussian_blobs((24, 24, 24), idx.astype(np.float64), 1.5, amps)
    assert np.abs(p.j[0] - ref).max() <= 1e-6 * ref.max()


@pytest.mark.gpu
def test_full_size_march(torch_cuda):
    """All 2097 sources, the default path (one bin: 64-bit fixed-point sums) against the oracle at the
    parity bar (rel-L2 <= 1e-5, max-abs-rel <= 1e-4); the 64-bit fixed-point mode too, and the
    sum over sources of separate fixed-point runs equals the whole. The sources sit in a few
    clusters of high-kappa cells, so the cells around a cluster and the clamped box corners take
    ~1e5 additions each, most far smaller than the sum they land on: FP32 reductions round many of
    them away (accumulation="fp32", measured rel-L2 ~1e-4, printed beside the others)."""
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.paper_timing()
    assert p.sources.shape == (2097, 3)
    ns = oracle.num_substeps(p.step_size, 1.0, p.time_step)
    j, k = (torch.from_numpy(a).cuda() for a in (p.j, p.kappa))
    s = torch.from_numpy(p.sources).cuda()

    def run(g, src):
        return g.advance(j, k, src, p.num_rays, p.step_size, 1.0, p.time_step).cpu().numpy().astype(np.float64)

    cores = len(os.sched_getaffinity(0))
    R = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns, threads=cores, ray_block=256)

    def errs(F):
        return np.linalg.norm(F - R) / np.linalg.norm(R), np.abs(F - R).max() / np.abs(R).max()

    g = Grid(p.shape, 1)
    F = run(g, s)
    assert g.last_accumulation() == "fixed"
    rel, mx = errs(F)
    print(f"default (fixed-point sums) vs oracle: rel-L2 {rel:.3e}, max-abs-rel {mx:.3e}")
    assert rel <= 1e-5 and mx <= 1e-4

    gt = Grid(p.shape, 1, autotune=True)
    Ft = run(gt, s)
    rel_t, mx_t = errs(Ft)
    print(f"autotuned ({gt.last_accumulation()}, {gt.last_plan()}) vs oracle: rel-L2 {rel_t:.3e}, max-abs-rel {mx_t:.3e}")
    assert rel_t <= 1e-5 and mx_t <= 1e-4

    gd = Grid(p.shape, 1, deterministic=True)
    exact = run(gd, s)
    halves = run(gd, s[:1000]) + run(gd, s[1000:])
    assert np.linalg.norm(exact - halves) <= 1e-6 * np.linalg.norm(exact)
    rel_d, mx_d = errs(exact)
    print(f"deterministic mode vs oracle: rel-L2 {rel_d:.3e}, max-abs-rel {mx_d:.3e}")
    assert rel_d <= 1e-5 and mx_d <= 1e-4

    g64 = Grid(p.shape, 1, accumulation="fp64")
    rel64, mx64 = errs(run(g64, s))
    print(f"FP64 sums vs oracle: rel-L2 {rel64:.3e}, max-abs-rel {mx64:.3e}")
    assert rel64 <= 1e-5 and mx64 <= 1e-4

    g32 = Grid(p.shape, 1, accumulation="fp32")
    rel32, mx32 = errs(run(g32, s))
    print(f"FP32 sums (opt-in) vs oracle: rel-L2 {rel32:.3e}, max-abs-rel {mx32:.3e}")
    assert rel32 <= 1e-3
