"""GPU parity with the round-to-nearest kappa convention (kappa_mode 1: kappa at the clamped
floor(x_k + 1/2), the other reading of the paper's nearest-cell kappa, Sec. 2) on every path
that carries its own kappa-cell code: each launch plan family, the batched persistent kernel,
the stateful advance, the reverse march and the source-position gradient; against the FP64
oracle run with the same convention.
"""
import numpy as np
import pytest

import oracle
from paper_2511_09389_gb300 import inputs

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
MAX_ABS_REL = 1e-4
GRAD_REL = 1e-3
PLANS = [None, (4, 32, 4), (4, 32, 0), (4, 32, 4, 2), (1, 64, 4, 2), (2, 64, 3), (1, 64, 1), (2, 32, 0, 2),
         (1, 32, 4), (2, 64, 2), (1, 64, 1, 1, 1), (4, 32, 0, 1, 1)]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2511_09389_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


def problem(seed, shape=(13, 11, 15), n_freq=4, num_rays=97, horizon=10.0):
    return inputs.random_small(seed, shape=shape, n_freq=n_freq, n_src=3, num_rays=num_rays, step_size=0.6,
                               horizon=horizon)


def ns_of(p):
    return oracle.num_substeps(p.step_size, p.radiation_velocity, p.time_step)


def assert_parity(F, R):
    F = np.asarray(F, np.float64).reshape(R.shape)
    for b in range(R.shape[0]):
        d = F[b] - R[b]
        e2 = np.linalg.norm(d) / np.linalg.norm(R[b])
        emax = np.abs(d).max() / np.abs(R[b]).max()
        assert e2 <= REL_L2 and emax <= MAX_ABS_REL, f"bin {b}: rel-L2 {e2:.3e}, max-abs-rel {emax:.3e}"


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def test_every_plan_family(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = problem(900)
    R = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns_of(p), kappa_mode=1)
    R0 = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns_of(p), kappa_mode=0)
    assert np.linalg.norm(R - R0) > 1e-4 * np.linalg.norm(R)      # the conventions differ here
    for plan in PLANS:
        g = Grid(p.shape, 8, kappa_mode=1, plan=plan)
        F = g.advance(dev(torch, p.j), dev(torch, p.kappa), dev(torch, p.sources), p.num_rays, p.step_size,
                      p.radiation_velocity, p.time_step)
        torch.cuda.synchronize()
        try:
            assert_parity(F.cpu().numpy(), R)
        except AssertionError as e:
            raise AssertionError(f"plan {plan}: {e}") from None
        g.close()


def test_batched_instances(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Batch
    probs = [problem(910 + i, shape=s, n_freq=nf, num_rays=nr) for i, (s, nf, nr) in
             enumerate([((13, 11, 15), 1, 97), ((9, 12, 10), 2, 150), ((16, 8, 12), 4, 61), ((7, 7, 7), 5, 200)])]
    inst = []
    for p in probs:
        d = {"j": dev(torch, p.j), "kappa": dev(torch, p.kappa), "sources": dev(torch, p.sources)}
        d.update(num_rays=p.num_rays, step_size=p.step_size, radiation_velocity=1.0, time_step=p.time_step)
        inst.append(d)
    b = Batch(inst, kappa_mode=1)
    outs = [o.cpu().numpy() for o in b.run()]
    torch.cuda.synchronize()
    b.close()
    for p, F in zip(probs, outs):
        assert_parity(F, oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns_of(p), kappa_mode=1))


def test_stateful_advance(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = problem(920, n_freq=3, horizon=4.0)
    g = Grid(p.shape, 8, kappa_mode=1)
    st = oracle.MarchState(p.n_freq, len(p.sources), p.num_rays)
    s = dev(torch, p.sources)
    for call, (aj, ak) in enumerate([(1.0, 1.0), (0.5, 1.7), (2.0, 0.3)]):
        j = (p.j * aj).astype(np.float32)
        k = (p.kappa * ak).astype(np.float32)
        F = g.advance_continue(dev(torch, j), dev(torch, k), s, p.num_rays, p.step_size, 1.0, p.time_step,
                               restart=(call == 0)).cpu().numpy()
        R = oracle.advance_state(j, k, p.sources, p.num_rays, p.step_size, ns_of(p), st, restart=(call == 0),
                                 kappa_mode=1)
        try:
            assert_parity(F, R)
        except AssertionError as e:
            raise AssertionError(f"call {call}: {e}") from None
    g.close()


@pytest.mark.parametrize("n_freq,stride", [(1, 4), (2, 8), (4, 16)])
def test_reverse_march_and_source_gradient(torch_cuda, n_freq, stride):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = problem(930 + n_freq, n_freq=n_freq)
    G = np.random.default_rng(n_freq).standard_normal(p.j.shape)
    g = Grid(p.shape, 8, kappa_mode=1, ckpt_stride=stride)
    gj, gk, gs = g.backward(dev(torch, G), dev(torch, p.j), dev(torch, p.kappa), dev(torch, p.sources), p.num_rays,
                            p.step_size, p.radiation_velocity, p.time_step, need_sources=True)
    torch.cuda.synchronize()
    gj, gk, gs = (a.cpu().numpy().astype(np.float64) for a in (gj, gk, gs))
    g.close()
    rj, rk = oracle.backward(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns_of(p), G, kappa_mode=1)
    rs = oracle.source_gradient(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns_of(p), G, kappa_mode=1)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    for b in range(n_freq):
        assert rel(gj[b], rj[b]) <= GRAD_REL and rel(gk[b], rk[b]) <= GRAD_REL, b
    assert rel(gs, rs) <= GRAD_REL
