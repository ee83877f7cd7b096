"""GPU parity at the largest grid the library accepts: 1024 x 1024 x 511 cells, whose packed
bin groups of four fill the 32-bit cell and element index to 2^31 - 2^22.

The FP64 oracle cannot run at this size, so the check is a property that holds at any size:
for uniform j and kappa every ray deposits (4 pi / N_Omega) sum_k (k+1) j ds exp(-kappa k ds)
in total (Eq. 2 with E_k = exp(-kappa k ds); clamped trilinear weights sum to one), so the
field summed over a box around one source equals that source's closed form when the sources
are farther apart than two light-travel radii. Sources next to the first and the last cells and
in the middle exercise the lowest and highest indices.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPE = (1024, 1024, 511)
SOURCES = [[6.3, 9.7, 4.2], [512.4, 511.8, 255.5], [1017.6, 1020.1, 506.9]]
NS, DS, J0 = 64, 0.5, 0.7
KAPPA = [0.05, 0.0, 0.1, 0.02]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2511_09389_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


def per_source(kap):
    k = np.arange(NS)
    return 4.0 * math.pi * float(np.sum((k + 1) * J0 * DS * np.exp(-kap * k * DS)))


def test_limit_is_the_largest_accepted_grid():
    """One more row along axis 2 crosses 2^31 and is refused (the CPU ABI test covers more)."""
    assert SHAPE[0] * SHAPE[1] * SHAPE[2] * 4 < 2 ** 31 <= SHAPE[0] * SHAPE[1] * (SHAPE[2] + 1) * 4


@pytest.mark.parametrize("n_freq,opts", [(1, {}), (4, {}), (4, {"accumulation": "fixed"})])
def test_largest_grid_closed_form_per_source(torch_cuda, n_freq, opts):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    g = Grid(SHAPE, n_freq, **opts)
    j = torch.full((n_freq,) + SHAPE, J0, dtype=torch.float32, device="cuda")
    kap = torch.empty_like(j)
    for b in range(n_freq):
        kap[b].fill_(KAPPA[b])
    s = torch.tensor(SOURCES, dtype=torch.float32, device="cuda")
    out = g.advance(j, kap, s, 512, DS, 1.0, NS * DS)
    torch.cuda.synchronize()
    del j, kap
    R = int(math.ceil(NS * DS)) + 2
    for b in range(n_freq):
        expect = per_source(KAPPA[b])
        total = out[b].sum(dtype=torch.float64).item()
        assert abs(total / (len(SOURCES) * expect) - 1) < 2e-5, (b, total)
        for src in SOURCES:
            lo = [max(0, int(math.floor(c)) - R) for c in src]
            hi = [min(n, int(math.floor(c)) + R + 2) for c, n in zip(src, SHAPE)]
            box = out[b, lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]].sum(dtype=torch.float64).item()
            assert abs(box / expect - 1) < 2e-5, (b, src, box, expect)
    # the cells next to the far corner hold deposits: the highest indices were written
    assert out[:, -3:, -3:, -3:].sum().item() > 0.0
    g.close()
    del out
    torch.cuda.empty_cache()
