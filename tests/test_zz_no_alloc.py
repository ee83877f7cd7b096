"""rt_advance_noalloc: the allocation-free forward march.

It is meant for callers that cannot allocate memory while they run (their GPU memory belongs
to another framework's pool or a fixed budget, or they must never block in an allocator).
Called through the C ABI, it must reproduce rt_advance on two calls in a row -- with different
grid shapes, bin counts and lattice sizes, so the shared static scratch is reused and its
stale contents must not leak -- and it must reject a problem larger than its scratch.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2511_09389_gb300 import inputs

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
MAX_ABS_REL = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2511_09389_gb300 import build, _native
    build.build()
    assert torch.cuda.is_available()
    return torch, _native.load()


def noalloc(torch, lib, p, out):
    j, k, s = (torch.from_numpy(a).cuda() for a in (p.j, p.kappa, p.sources))
    n0, n1, n2 = p.shape
    st = lib.rt_advance_noalloc(j.data_ptr(), k.data_ptr(), s.data_ptr(), s.shape[0], n0, n1, n2, p.num_rays,
                                p.step_size, p.radiation_velocity, p.time_step, p.n_freq, out.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    return st, (j, k, s)


def reference(torch, p):
    from paper_2511_09389_gb300.api import Grid
    g = Grid(p.shape, 8)
    j, k, s = (torch.from_numpy(a).cuda() for a in (p.j, p.kappa, p.sources))
    out = g.advance(j, k, s, p.num_rays, p.step_size, p.radiation_velocity, p.time_step)
    torch.cuda.synchronize()
    res = out.cpu().numpy().astype(np.float64)
    g.close()
    return res


def close(F, R):
    for b in range(R.shape[0]):
        rel = np.linalg.norm(F[b] - R[b]) / np.linalg.norm(R[b])
        mx = np.abs(F[b] - R[b]).max() / np.abs(R[b]).max()
        assert rel <= REL_L2 and mx <= MAX_ABS_REL, (b, rel, mx)


def test_noalloc_matches_advance_on_consecutive_calls(env):
    torch, lib = env
    a = inputs.random_small(71, shape=(32, 30, 28), n_freq=4, n_src=5, num_rays=768, horizon=24.0)
    b = inputs.random_small(72, shape=(24, 20, 36), n_freq=3, n_src=3, num_rays=300, step_size=0.6,
                            horizon=20.0)
    outs = []
    for p in (a, b):
        out = torch.full(p.j.shape, float("nan"), device="cuda")
        st, keep = noalloc(torch, lib, p, out)
        assert st == 0, lib.rt_last_error().decode()
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy().astype(np.float64))
    close(outs[0], reference(torch, a))
    close(outs[1], reference(torch, b))
    # the same inputs again after a different problem: stale scratch must not leak in
    out = torch.empty(a.j.shape, device="cuda")
    st, keep = noalloc(torch, lib, a, out)
    assert st == 0
    torch.cuda.synchronize()
    close(out.cpu().numpy().astype(np.float64), outs[0])


def test_noalloc_single_bin_and_rejects_oversize(env):
    torch, lib = env
    p = inputs.single_source_uniform(n=24, num_rays=500, horizon=10.0)
    out = torch.empty(p.j.shape, device="cuda")
    st, keep = noalloc(torch, lib, p, out)
    assert st == 0
    torch.cuda.synchronize()
    close(out.cpu().numpy().astype(np.float64), reference(torch, p))
    # 96^3 with 4 bins needs 3 x 13.5 MiB of packed scratch: more than the static array holds
    big = inputs.Problem("big", np.zeros((4, 96, 96, 96), np.float32), np.zeros((4, 96, 96, 96), np.float32),
                         np.zeros((1, 3), np.float32), 64, 0.5, 1.0, 4.0)
    out = torch.empty(big.j.shape, device="cuda")
    st, keep = noalloc(torch, lib, big, out)
    assert st == 1 and b"static scratch" in lib.rt_last_error()
    many_rays = inputs.single_source_uniform(n=8, num_rays=20000, horizon=2.0)
    out = torch.empty(many_rays.j.shape, device="cuda")
    st, keep = noalloc(torch, lib, many_rays, out)
    assert st == 1 and b"rays" in lib.rt_last_error()


def test_noalloc_matches_oracle_and_allocates_nothing(env):
    """Directly against the FP64 oracle (not only through rt_advance), and the property the entry
    point exists for: after a warm-up call on this device (which commits the static array and
    loads the kernels), further calls leave the device's free memory unchanged -- nothing is
    allocated, by the library or by the CUDA runtime on its behalf."""
    import oracle
    torch, lib = env
    p = inputs.random_small(73, shape=(20, 18, 22), n_freq=4, n_src=4, num_rays=500, horizon=16.0)
    out = torch.empty(p.j.shape, device="cuda")
    st, keep = noalloc(torch, lib, p, out)                 # warm-up: commits the scratch, loads kernels
    assert st == 0, lib.rt_last_error().decode()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    j, k, s = keep
    n0, n1, n2 = p.shape
    for _ in range(3):
        st = lib.rt_advance_noalloc(j.data_ptr(), k.data_ptr(), s.data_ptr(), s.shape[0], n0, n1, n2, p.num_rays,
                                    p.step_size, p.radiation_velocity, p.time_step, p.n_freq, out.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
        assert st == 0, lib.rt_last_error().decode()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0
    R = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size,
                       oracle.num_substeps(p.step_size, p.radiation_velocity, p.time_step))
    close(out.cpu().numpy().astype(np.float64), R)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 9, 11), (9, 11, 1), (7, 2, 1), (2, 2, 2)])
def test_noalloc_on_degenerate_extents(env, shape):
    """Slab, line and single-cell grids through the allocation-free entry point, against the
    FP64 oracle."""
    import oracle
    torch, lib = env
    p = inputs.random_small(90 + sum(shape), shape=shape, n_freq=3, n_src=3, num_rays=37, step_size=0.6,
                            horizon=9.0)
    out = torch.empty(p.j.shape, device="cuda")
    st, _ = noalloc(torch, lib, p, out)
    assert st == 0, lib.rt_last_error().decode()
    torch.cuda.synchronize()
    R = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size,
                       oracle.num_substeps(p.step_size, p.radiation_velocity, p.time_step))
    close(out.cpu().numpy().astype(np.float64), R)
