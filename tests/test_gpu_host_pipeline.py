"""Pipelined host-buffer advance (rt_advance_host_async / rt_host_wait / rt_host_join).

Consecutive enqueued calls with different inputs land, in order, in their own host buffers and
equal the same calls made one at a time (bitwise in the deterministic mode, against the oracle in
FP32); a change of problem size drains and regrows the buffer sets; two calls sharing one output
buffer leave the later field there; a stream joined to the pipeline sees the finished copies.
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


def pinned(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()


def test_enqueued_calls_equal_single_calls_bitwise(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.random_small(31, shape=(20, 18, 22), n_freq=3, n_src=3, num_rays=192, step_size=0.5, horizon=8.0)
    g = Grid(p.shape, 4, deterministic=True)
    scales = [(1.0, 1.0), (0.5, 2.0), (3.0, 0.25), (1.5, 1.0), (0.2, 0.7)]
    js = [pinned(torch, p.j * a) for a, _ in scales]
    ks = [pinned(torch, p.kappa * b) for _, b in scales]
    srcs = pinned(torch, p.sources)
    outs = [torch.empty(js[0].shape, dtype=torch.float32).pin_memory() for _ in scales]
    for jh, kh, oh in zip(js, ks, outs):
        g.advance_host_async(jh, kh, srcs, p.num_rays, p.step_size, 1.0, p.time_step, out=oh)
    g.host_wait()
    ref = Grid(p.shape, 4, deterministic=True)
    s = srcs.cuda()
    for jh, kh, oh in zip(js, ks, outs):
        want = ref.advance(jh.cuda(), kh.cuda(), s, p.num_rays, p.step_size, 1.0, p.time_step).cpu()
        assert torch.equal(oh, want)


def test_fp32_pipeline_matches_the_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.random_small(32, shape=(16, 24, 20), n_freq=4, n_src=2, num_rays=256, step_size=0.5, horizon=9.0)
    g = Grid(p.shape, 8)
    ns = oracle.num_substeps(p.step_size, 1.0, p.time_step)
    cases = [(1.0, 1.0), (2.0, 0.5), (0.7, 1.3)]
    js = [pinned(torch, p.j * a) for a, _ in cases]
    ks = [pinned(torch, p.kappa * b) for _, b in cases]
    srcs = pinned(torch, p.sources)
    outs = [torch.empty(js[0].shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    results = []
    for i, (jh, kh) in enumerate(zip(js, ks)):
        g.advance_host_async(jh, kh, srcs, p.num_rays, p.step_size, 1.0, p.time_step, out=outs[i & 1])
        if i & 1:
            g.host_wait()
            results += [outs[0].numpy().copy(), outs[1].numpy().copy()]
    g.host_wait()
    results.append(outs[0].numpy().copy())
    for (jh, kh), F in zip(zip(js, ks), results):
        R = oracle.advance(jh.numpy(), kh.numpy(), p.sources, p.num_rays, p.step_size, ns)
        F = F.astype(np.float64).reshape(R.shape[0], -1)
        R = R.reshape(R.shape[0], -1)
        for b in range(R.shape[0]):
            e2 = np.linalg.norm(F[b] - R[b]) / np.linalg.norm(R[b])
            emax = np.abs(F[b] - R[b]).max() / np.abs(R[b]).max()
            assert e2 <= 1e-5 and emax <= 1e-4, (b, e2, emax)


def test_size_change_and_shared_output(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.random_small(33, shape=(12, 14, 10), n_freq=4, n_src=2, num_rays=128, step_size=0.5, horizon=6.0)
    g = Grid(p.shape, 4, deterministic=True)
    srcs = pinned(torch, p.sources)
    one_j, one_k = pinned(torch, p.j[:1]), pinned(torch, p.kappa[:1])
    all_j, all_k = pinned(torch, p.j), pinned(torch, p.kappa)
    o1 = torch.empty(one_j.shape, dtype=torch.float32).pin_memory()
    o4 = torch.empty(all_j.shape, dtype=torch.float32).pin_memory()
    # one bin, then four bins (the buffer sets grow while the first call may be in flight)
    g.advance_host_async(one_j, one_k, srcs, p.num_rays, p.step_size, 1.0, p.time_step, out=o1)
    g.advance_host_async(all_j, all_k, srcs, p.num_rays, p.step_size, 1.0, p.time_step, out=o4)
    g.host_wait()
    ref = Grid(p.shape, 4, deterministic=True)
    s = srcs.cuda()
    want4 = ref.advance(all_j.cuda(), all_k.cuda(), s, p.num_rays, p.step_size, 1.0, p.time_step).cpu()
    assert torch.equal(o4, want4)
    want1 = ref.advance(one_j.cuda(), one_k.cuda(), s, p.num_rays, p.step_size, 1.0, p.time_step).cpu()
    assert torch.equal(o1, want1)
    # two calls into one output buffer: the later field stays
    half_j = pinned(torch, p.j * 0.5)
    g.advance_host_async(all_j, all_k, srcs, p.num_rays, p.step_size, 1.0, p.time_step, out=o4)
    g.advance_host_async(half_j, all_k, srcs, p.num_rays, p.step_size, 1.0, p.time_step, out=o4)
    g.host_wait()
    want_half = ref.advance(half_j.cuda(), all_k.cuda(), s, p.num_rays, p.step_size, 1.0, p.time_step).cpu()
    assert torch.equal(o4, want_half)


def test_join_orders_a_stream_after_the_copies(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.random_small(34, shape=(16, 16, 16), n_freq=2, n_src=2, num_rays=160, step_size=0.5, horizon=7.0)
    g = Grid(p.shape, 2, deterministic=True)
    jh, kh, sh = pinned(torch, p.j), pinned(torch, p.kappa), pinned(torch, p.sources)
    out = torch.empty(jh.shape, dtype=torch.float32).pin_memory()
    side = torch.cuda.Stream()
    g.advance_host_async(jh, kh, sh, p.num_rays, p.step_size, 1.0, p.time_step, out=out)
    g.host_join(side)
    done = torch.cuda.Event()
    done.record(side)
    done.synchronize()
    want = Grid(p.shape, 2, deterministic=True).advance(jh.cuda(), kh.cuda(), sh.cuda(), p.num_rays,
                                                         p.step_size, 1.0, p.time_step).cpu()
    assert torch.equal(out, want)
    g.host_wait()
    g.host_wait()   # nothing left: returns at once


def test_rejects_bad_arguments_before_enqueueing(torch_cuda):
    """NULL buffers and bad scalars return INVALID_ARG with nothing enqueued; the handle's next
    pipelined call still works."""
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid, RTError
    g = Grid((8, 8, 8), 1, deterministic=True)
    st = g._lib.rt_advance_host_async(g._h, None, None, None, 0, 16, 0.5, 1.0, 2.0, 1, None, None)
    assert st == 1   # RT_ERR_INVALID_ARG
    assert g._lib.rt_host_wait(g._h) == 0
    p = inputs.random_small(35, shape=(8, 8, 8), n_freq=1, n_src=2, num_rays=64, step_size=0.5, horizon=4.0)
    jh, kh, sh = pinned(torch, p.j), pinned(torch, p.kappa), pinned(torch, p.sources)
    out = torch.empty(jh.shape, dtype=torch.float32).pin_memory()
    for bad in (dict(num_rays=0), dict(step_size=0.0), dict(time_step=-1.0)):
        kw = dict(num_rays=p.num_rays, step_size=p.step_size, time_step=p.time_step)
        kw.update(bad)
        with pytest.raises(RTError, match="INVALID_ARG"):
            g.advance_host_async(jh, kh, sh, kw["num_rays"], kw["step_size"], 1.0, kw["time_step"], out=out)
    g.host_wait()
    g.advance_host_async(jh, kh, sh, p.num_rays, p.step_size, 1.0, p.time_step, out=out)
    g.host_wait()
    want = Grid(p.shape, 1, deterministic=True).advance(jh.cuda(), kh.cuda(), sh.cuda(), p.num_rays,
                                                        p.step_size, 1.0, p.time_step).cpu()
    assert torch.equal(out, want)
