"""GPU parity on degenerate grids: extents of one or two cells (slabs, lines, a single cell),
through the C ABI, against the FP64 oracle (itself pinned on these shapes in
test_oracle_degenerate.py). Every launch plan family, every accumulation, the reverse march
and the batched persistent kernel meet the same bars as on regular grids.
"""
import numpy as np
import pytest

import oracle
from paper_2511_09389_gb300 import inputs

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
MAX_ABS_REL = 1e-4
GRAD_REL = 1e-3

SHAPES = [(1, 1, 1), (1, 9, 11), (9, 1, 11), (9, 11, 1), (2, 7, 5), (7, 2, 1), (1, 2, 2), (2, 2, 2)]
PLANS = [None, (4, 32, 4), (4, 32, 0), (4, 32, 4, 2), (1, 64, 4, 2), (2, 64, 3), (1, 64, 1), (2, 32, 0, 2),
         (1, 32, 4)]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2511_09389_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


def problem(shape, seed, n_freq=4):
    return inputs.random_small(seed, shape=shape, n_freq=n_freq, n_src=3, num_rays=37, step_size=0.6,
                               horizon=9.0)


def oracle_field(p):
    ns = oracle.num_substeps(p.step_size, p.radiation_velocity, p.time_step)
    return oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns)


def assert_parity(F, R):
    F = np.asarray(F, np.float64).reshape(R.shape)
    for b in range(R.shape[0]):
        d = F[b] - R[b]
        e2 = np.linalg.norm(d) / np.linalg.norm(R[b])
        emax = np.abs(d).max() / np.abs(R[b]).max()
        assert e2 <= REL_L2 and emax <= MAX_ABS_REL, f"bin {b}: rel-L2 {e2:.3e}, max-abs-rel {emax:.3e}"


def advance(torch, p, **opts):
    from paper_2511_09389_gb300.api import Grid
    g = Grid(p.shape, 8, **opts)
    t = lambda a: torch.from_numpy(a).cuda()
    out = g.advance(t(p.j), t(p.kappa), t(p.sources), p.num_rays, p.step_size, p.radiation_velocity, p.time_step)
    torch.cuda.synchronize()
    F = out.cpu().numpy()
    g.close()
    return F


@pytest.mark.parametrize("shape", SHAPES)
def test_every_plan_family_on_degenerate_extents(torch_cuda, shape):
    p = problem(shape, 700 + sum(shape))
    R = oracle_field(p)
    for plan in PLANS:
        F = advance(torch_cuda, p, plan=plan)
        try:
            assert_parity(F, R)
        except AssertionError as e:
            raise AssertionError(f"plan {plan}: {e}") from None
    # the autotuner times every candidate (tiled ones included, which such grids cannot take)
    assert_parity(advance(torch_cuda, p, autotune=True), R)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 9, 11), (7, 2, 1), (2, 2, 2)])
def test_every_accumulation_on_degenerate_extents(torch_cuda, shape):
    p = problem(shape, 720 + sum(shape), n_freq=3)
    R = oracle_field(p)
    for opts in ({"accumulation": "fp32"}, {"accumulation": "fp64"}, {"accumulation": "fixed"},
                 {"deterministic": True}, {"kappa_mode": 0, "accumulation": "auto"}):
        assert_parity(advance(torch_cuda, p, **opts), R)
    # deterministic mode is bitwise reproducible here too
    a = advance(torch_cuda, p, deterministic=True)
    b = advance(torch_cuda, p, deterministic=True)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("shape,n_freq,stride", [((1, 9, 11), 1, 4), ((9, 11, 1), 2, 8), ((7, 2, 1), 1, 16),
                                                 ((1, 1, 1), 1, 4), ((2, 2, 2), 4, 8), ((9, 1, 11), 3, 32)])
def test_adjoint_on_degenerate_extents(torch_cuda, shape, n_freq, stride):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = problem(shape, 740 + sum(shape) + n_freq, n_freq=n_freq)
    G = np.random.default_rng(n_freq + stride).standard_normal(p.j.shape)
    g = Grid(p.shape, 8, ckpt_stride=stride)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    gj, gk = g.backward(t(G), t(p.j), t(p.kappa), t(p.sources), p.num_rays, p.step_size,
                        p.radiation_velocity, p.time_step)
    torch.cuda.synchronize()
    gj, gk = gj.cpu().numpy(), gk.cpu().numpy()
    g.close()
    ns = oracle.num_substeps(p.step_size, p.radiation_velocity, p.time_step)
    rj, rk = oracle.backward(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns, G)
    for b in range(n_freq):
        for got, ref in ((gj[b], rj[b]), (gk[b], rk[b])):
            e = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert e <= GRAD_REL, (b, e)


def test_batch_of_degenerate_instances(torch_cuda):
    """The batched persistent kernel on slab, line and single-cell instances."""
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Batch
    probs = [problem(s, 760 + i, n_freq=nf) for i, (s, nf) in
             enumerate([((1, 9, 11), 1), ((7, 2, 1), 2), ((1, 1, 1), 4), ((2, 2, 2), 3), ((9, 11, 1), 5)])]
    dev = []
    for p in probs:
        d = {k: torch.from_numpy(v).cuda() for k, v in (("j", p.j), ("kappa", p.kappa), ("sources", p.sources))}
        d.update(num_rays=p.num_rays, step_size=p.step_size, radiation_velocity=1.0, time_step=p.time_step)
        dev.append(d)
    b = Batch(dev)
    outs = [o.cpu().numpy() for o in b.run()]
    torch.cuda.synchronize()
    b.close()
    for p, F in zip(probs, outs):
        assert_parity(F, oracle_field(p))


@pytest.mark.parametrize("num_rays,ns", [(1, 1), (1, 7), (2, 1), (2, 2), (33, 1), (5, 2)])
def test_fewest_rays_and_substeps(torch_cuda, num_rays, ns):
    """One ray (the lattice's single direction), two rays, and marches of one or two substeps
    (a ray's only corner set is flushed at the end), for every plan family."""
    p = inputs.random_small(780 + num_rays + ns, shape=(9, 7, 8), n_freq=4, n_src=3, num_rays=num_rays,
                            step_size=0.6, horizon=ns * 0.6)
    assert oracle.num_substeps(p.step_size, p.radiation_velocity, p.time_step) == ns
    R = oracle_field(p)
    for plan in PLANS:
        F = advance(torch_cuda, p, plan=plan)
        try:
            assert_parity(F, R)
        except AssertionError as e:
            raise AssertionError(f"plan {plan}: {e}") from None


@pytest.mark.parametrize("num_rays,ns,stride", [(1, 1, 4), (1, 7, 4), (2, 2, 8), (5, 3, 16)])
def test_adjoint_fewest_rays_and_substeps(torch_cuda, num_rays, ns, stride):
    """The reverse march when a ray has fewer substeps than one checkpoint segment."""
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    for n_freq in (1, 4):
        p = inputs.random_small(800 + num_rays + ns, shape=(9, 7, 8), n_freq=n_freq, n_src=3,
                                num_rays=num_rays, step_size=0.6, horizon=ns * 0.6)
        G = np.random.default_rng(ns).standard_normal(p.j.shape)
        g = Grid(p.shape, 8, ckpt_stride=stride)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
        gj, gk = g.backward(t(G), t(p.j), t(p.kappa), t(p.sources), p.num_rays, p.step_size,
                            p.radiation_velocity, p.time_step)
        torch.cuda.synchronize()
        gj, gk = gj.cpu().numpy(), gk.cpu().numpy()
        g.close()
        rj, rk = oracle.backward(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns, G)
        for b in range(n_freq):
            for got, ref in ((gj[b], rj[b]), (gk[b], rk[b])):
                if not np.any(ref):   # N_s = 1: I_0 = 0 and no later emission, so dL/dkappa = 0
                    assert not np.any(got), (n_freq, b)
                    continue
                e = np.linalg.norm(got - ref) / np.linalg.norm(ref)
                assert e <= GRAD_REL, (n_freq, b, e)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 9, 11), (7, 2, 1), (2, 2, 2)])
def test_stateful_advance_on_degenerate_extents(torch_cuda, shape):
    """rt_advance_continue (rays carried between calls, media changing between them) against the
    oracle's stateful advance on slab, line and single-cell grids."""
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.random_small(820 + sum(shape), shape=shape, n_freq=3, n_src=3, num_rays=41, step_size=0.5,
                            horizon=3.0)
    g = Grid(p.shape, 8)
    st = oracle.MarchState(p.n_freq, len(p.sources), p.num_rays)
    s = torch.from_numpy(p.sources).cuda()
    ns = oracle.num_substeps(p.step_size, 1.0, p.time_step)
    for call, (aj, ak) in enumerate([(1.0, 1.0), (0.5, 1.7), (2.0, 0.3)]):
        j = (p.j * aj).astype(np.float32)
        k = (p.kappa * ak).astype(np.float32)
        F = g.advance_continue(torch.from_numpy(j).cuda(), torch.from_numpy(k).cuda(), s, p.num_rays, p.step_size,
                               1.0, p.time_step, restart=(call == 0)).cpu().numpy()
        R = oracle.advance_state(j, k, p.sources, p.num_rays, p.step_size, ns, st, restart=(call == 0))
        try:
            assert_parity(F, R)
        except AssertionError as e:
            raise AssertionError(f"call {call}: {e}") from None
    g.close()


@pytest.mark.parametrize("shape,n_freq,stride", [((10, 1, 9), 1, 4), ((1, 9, 11), 2, 8), ((7, 2, 1), 4, 16),
                                                 ((1, 1, 1), 1, 4)])
def test_source_gradient_on_degenerate_extents(torch_cuda, shape, n_freq, stride):
    """rt_backward_sources against the oracle; along a single-cell axis the component vanishes."""
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = problem(shape, 840 + sum(shape) + n_freq, n_freq=n_freq)
    G = np.random.default_rng(n_freq + 3).standard_normal(p.j.shape)
    g = Grid(p.shape, 8, ckpt_stride=stride)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    _, _, gs = g.backward(t(G), t(p.j), t(p.kappa), t(p.sources), p.num_rays, p.step_size,
                          p.radiation_velocity, p.time_step, need_sources=True)
    torch.cuda.synchronize()
    gs = gs.cpu().numpy().astype(np.float64)
    g.close()
    ns = oracle.num_substeps(p.step_size, p.radiation_velocity, p.time_step)
    rs = oracle.source_gradient(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns, G)
    # the gradient's natural size: max |G| times max |F| per unit of length
    scale = np.abs(G).max() * np.abs(oracle_field(p)).max()
    if np.abs(rs).max() > 1e-9 * scale:          # a 1 x 1 x 1 grid has none: F does not move
        assert np.linalg.norm(gs - rs) / np.linalg.norm(rs) <= GRAD_REL
    for a, n in enumerate(shape):
        if n == 1:
            assert np.abs(gs[:, a]).max() <= 1e-6 * scale, (a, gs[:, a])
