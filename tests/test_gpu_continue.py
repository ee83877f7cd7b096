"""Stateful advance (rt_advance_continue): the march continued across calls.

Each call against the oracle's stateful advance on the same inputs (j and kappa change between
calls), the full-size workload split into four calls against one call over all substeps,
restarts (explicit, and implied by a new problem shape), zero-substep calls, and the refusal in
deterministic mode.
"""
import numpy as np
import pytest

import oracle
from paper_2511_09389_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2511_09389_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


def rel_errors(F, R):
    F = np.asarray(F, np.float64).reshape(R.shape[0], -1)
    R = R.reshape(R.shape[0], -1)
    return [(np.linalg.norm(F[b] - R[b]) / np.linalg.norm(R[b]), np.abs(F[b] - R[b]).max() / np.abs(R[b]).max())
            for b in range(R.shape[0])]


@pytest.mark.parametrize("plan", [None, (1, 32, 1, 1, 1), (4, 64, 0, 1, 0), (2, 32, 2, 1, 1), (4, 32, 0, 2)])
def test_calls_match_the_oracle_with_changing_media(torch_cuda, plan):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.random_small(21, shape=(14, 12, 16), n_freq=5, n_src=3, num_rays=160, step_size=0.5, horizon=5.0)
    g = Grid(p.shape, 8, plan=plan)
    st = oracle.MarchState(p.n_freq, len(p.sources), p.num_rays)
    s = torch.from_numpy(p.sources).cuda()
    ns = oracle.num_substeps(p.step_size, 1.0, p.time_step)
    for call, (aj, ak) in enumerate([(1.0, 1.0), (0.5, 1.7), (2.0, 0.3)]):
        j = (p.j * aj).astype(np.float32)
        k = (p.kappa * ak).astype(np.float32)
        F = g.advance_continue(torch.from_numpy(j).cuda(), torch.from_numpy(k).cuda(), s, p.num_rays, p.step_size,
                               1.0, p.time_step, restart=(call == 0)).cpu().numpy()
        R = oracle.advance_state(j, k, p.sources, p.num_rays, p.step_size, ns, st, restart=(call == 0))
        for b, (e2, emax) in enumerate(rel_errors(F, R)):
            assert e2 <= 1e-5 and emax <= 1e-4, (call, b, e2, emax)
    assert g.last_plan()["lanes_per_ray"] == 1


def test_four_calls_equal_one_call_full_size(torch_cuda):
    """The benchmark workload (128^3, 16 sources, N_Omega 3072, 4 bins): four calls of c dt 32
    add up to one call of c dt 128 (N_s 64 x 4 = 256)."""
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.turbulent()
    j, k, s = (torch.from_numpy(a).cuda() for a in (p.j, p.kappa, p.sources))
    g = Grid(p.shape, 8)
    total = torch.zeros_like(j)
    for call in range(4):
        g.advance_continue(j, k, s, p.num_rays, p.step_size, 1.0, 32.0, out=total, accumulate=call > 0,
                           restart=call == 0)
    one = g.advance(j, k, s, p.num_rays, p.step_size, 1.0, 128.0)
    a, b = total.double().cpu().numpy(), one.double().cpu().numpy()
    for e2, emax in rel_errors(a, b):
        assert e2 <= 1e-5 and emax <= 1e-4


def test_restart_and_new_shapes_start_at_the_sources(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.random_small(22, shape=(12, 12, 12), n_freq=2, n_src=2, num_rays=96, step_size=0.5, horizon=4.0)
    j, k, s = (torch.from_numpy(a).cuda() for a in (p.j, p.kappa, p.sources))
    g = Grid(p.shape, 8)
    fresh = g.advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step).cpu().numpy()
    for _ in range(2):
        g.advance_continue(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
    again = g.advance_continue(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step, restart=True).cpu().numpy()
    assert max(e for e, _ in rel_errors(again, fresh.astype(np.float64))) <= 1e-6
    # a different ray count is another problem: the rays start over
    fresh2 = g.advance(j, k, s, 64, p.step_size, 1.0, p.time_step).cpu().numpy()
    other = g.advance_continue(j, k, s, 64, p.step_size, 1.0, p.time_step).cpu().numpy()
    assert max(e for e, _ in rel_errors(other, fresh2.astype(np.float64))) <= 1e-6


def test_zero_substep_call_keeps_the_state(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.random_small(23, shape=(12, 10, 14), n_freq=1, n_src=2, num_rays=128, step_size=0.5, horizon=4.0)
    j, k, s = (torch.from_numpy(a).cuda() for a in (p.j, p.kappa, p.sources))
    g = Grid(p.shape, 8)
    a = g.advance_continue(j, k, s, p.num_rays, p.step_size, 1.0, 4.0, restart=True).cpu().numpy()
    z = g.advance_continue(j, k, s, p.num_rays, p.step_size, 1.0, 0.0).cpu().numpy()
    assert not np.any(z)
    b = g.advance_continue(j, k, s, p.num_rays, p.step_size, 1.0, 4.0).cpu().numpy()
    one = g.advance(j, k, s, p.num_rays, p.step_size, 1.0, 8.0).cpu().numpy().astype(np.float64)
    assert max(e for e, _ in rel_errors(a.astype(np.float64) + b, one)) <= 1e-5


def test_deterministic_handle_refuses(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid, RTError
    g = Grid((8, 8, 8), 1, deterministic=True)
    j = torch.ones(1, 8, 8, 8, device="cuda")
    s = torch.full((1, 3), 3.5, device="cuda")
    with pytest.raises(RTError, match="UNSUPPORTED"):
        g.advance_continue(j, j, s, 16, 0.5, 1.0, 2.0)
