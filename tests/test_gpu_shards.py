"""Direction shards (rt_advance_rays, Sec. 2: directions split across devices, partial fields
summed) for every launch plan family: ragged shards of the lattice, one ray, empty ranges,
added into one field, equal the whole advance and the FP64 oracle; each shard equals the
oracle run on the same ray range."""
import numpy as np
import pytest

import oracle
from paper_2511_09389_gb300 import inputs

pytestmark = pytest.mark.gpu

PLANS = [None, (4, 32, 4), (4, 32, 0), (4, 32, 4, 2), (1, 64, 4, 2), (2, 64, 3), (1, 64, 1), (2, 32, 0, 2),
         (1, 32, 4), (1, 64, 1, 1, 1), (4, 32, 0, 1, 1)]
SHARDS = [(0, 1), (1, 34), (34, 34), (34, 96), (96, 97), (97, 131)]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2511_09389_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


def rel_errors(F, R):
    out = []
    for b in range(R.shape[0]):
        d = np.asarray(F[b], np.float64) - R[b]
        out.append((np.linalg.norm(d) / np.linalg.norm(R[b]), np.abs(d).max() / np.abs(R[b]).max()))
    return out


@pytest.mark.parametrize("plan", PLANS)
def test_ragged_shards_sum_to_the_whole(torch_cuda, plan):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.random_small(950, shape=(14, 12, 16), n_freq=4, n_src=3, num_rays=131, step_size=0.6, horizon=8.0)
    assert SHARDS[-1][1] == p.num_rays
    ns = oracle.num_substeps(p.step_size, p.radiation_velocity, p.time_step)
    g = Grid(p.shape, 8, plan=plan, accumulation="fp32")
    j, k, s = (torch.from_numpy(a).cuda() for a in (p.j, p.kappa, p.sources))
    acc = torch.zeros(p.j.shape, device="cuda")
    for rb, re in SHARDS:
        g.advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step, out=acc, accumulate=True, ray_range=(rb, re))
        if re - rb >= 30:
            one = g.advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step, ray_range=(rb, re))
            R = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns, ray_range=(rb, re))
            for e2, emax in rel_errors(one.cpu().numpy(), R):
                assert e2 <= 1e-5 and emax <= 1e-4, (plan, rb, re, e2, emax)
    torch.cuda.synchronize()
    R = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns)
    for e2, emax in rel_errors(acc.cpu().numpy(), R):
        assert e2 <= 1e-5 and emax <= 1e-4, (plan, e2, emax)
    g.close()
