"""GPU reverse-march adjoint (rt_backward) against the FP64 oracle's adjoint and FP64 finite
differences; the autograd wrapper; gradient-based inversion (Sec. 4).

Bar: relative L2 error of dL/dj and dL/dkappa <= 1e-3 per bin against the oracle adjoint
(itself pinned to FP64 central differences in test_oracle_pins.py) and against GPU-side
directional finite differences evaluated in FP64 by the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2511_09389_gb300 import inputs

pytestmark = pytest.mark.gpu

GRAD_REL = 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2511_09389_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def gpu_backward(torch, p, G, **opts):
    from paper_2511_09389_gb300.api import Grid
    g = Grid(p.shape, 8, **opts)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    gj, gk = g.backward(t(G), t(p.j), t(p.kappa), t(p.sources), p.num_rays, p.step_size,
                        p.radiation_velocity, p.time_step)
    torch.cuda.synchronize()
    return gj.cpu().numpy(), gk.cpu().numpy()


def oracle_backward(p, G, kappa_mode=0):
    ns = oracle.num_substeps(p.step_size, p.radiation_velocity, p.time_step)
    return oracle.backward(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns, G, kappa_mode=kappa_mode)


@pytest.mark.parametrize("n_freq,stride", [(1, 4), (1, 8), (1, 16), (2, 4), (2, 16), (3, 32), (4, 4), (4, 8), (5, 16)])
def test_adjoint_matches_oracle(torch_cuda, n_freq, stride):
    p = inputs.random_small(100 + n_freq, shape=(14, 11, 17), n_freq=n_freq, n_src=4, num_rays=97,
                            step_size=0.6, horizon=15.0)   # N_s = 25: ragged last segment
    G = np.random.default_rng(n_freq).standard_normal(p.j.shape)
    gj, gk = gpu_backward(torch_cuda, p, G, ckpt_stride=stride)
    rj, rk = oracle_backward(p, G)
    for b in range(n_freq):
        assert rel(gj[b], rj[b]) <= GRAD_REL, (b, rel(gj[b], rj[b]))
        assert rel(gk[b], rk[b]) <= GRAD_REL, (b, rel(gk[b], rk[b]))


def test_adjoint_kappa_mode_round(torch_cuda):
    p = inputs.random_small(120, shape=(12, 12, 12), n_freq=4, n_src=3, num_rays=150, horizon=12.0)
    G = np.random.default_rng(3).standard_normal(p.j.shape)
    gj, gk = gpu_backward(torch_cuda, p, G, kappa_mode=1)
    rj, rk = oracle_backward(p, G, kappa_mode=1)
    assert rel(gj, rj) <= GRAD_REL and rel(gk, rk) <= GRAD_REL


def test_adjoint_vs_central_fd_16cubed(torch_cuda):
    """dL/dkappa and dL/dj against FP64 central differences (h = 1e-6) on a 16^3 lognormal
    medium with N_Omega = 192, L = <G, F>: the GPU adjoint's directional derivatives."""
    n = 16
    kap = inputs.lognormal_field((n, n, n), 1.0, 0.05, 41)[None]
    src = np.array([[7.3, 8.1, 6.6], [3.0, 11.5, 9.2]], np.float32)
    j = inputs.gaussian_blobs((n, n, n), src, 2.0, [1.0, 0.6])[None]
    p = inputs.Problem("fd", j, kap, src, 192, 0.5, 1.0, 10.0)
    ns = 20
    rng = np.random.default_rng(4)
    G = rng.standard_normal(j.shape)
    gj, gk = gpu_backward(torch_cuda, p, G)
    h = 1e-6
    for target in ("kappa", "j"):
        for _ in range(3):
            e = rng.standard_normal(j.shape)
            jj, kk = (j.astype(np.float64), kap.astype(np.float64))
            if target == "kappa":
                Fp = oracle.advance(jj, kk + h * e, src, 192, 0.5, ns)
                Fm = oracle.advance(jj, kk - h * e, src, 192, 0.5, ns)
                ad = np.sum(gk * e)
            else:
                Fp = oracle.advance(jj + h * e, kk, src, 192, 0.5, ns)
                Fm = oracle.advance(jj - h * e, kk, src, 192, 0.5, ns)
                ad = np.sum(gj * e)
            fd = (np.sum(G * Fp) - np.sum(G * Fm)) / (2 * h)
            assert abs(ad - fd) <= GRAD_REL * abs(fd), (target, ad, fd)


def test_adjoint_full_size_inverse_workload(torch_cuda):
    """64^3 lognormal, 8 sources at blob centres, N_Omega 3072, N_s 128, one bin."""
    p = inputs.inverse_problem()
    G = np.random.default_rng(8).standard_normal(p.j.shape)
    gj, gk = gpu_backward(torch_cuda, p, G)
    rj, rk = oracle_backward(p, G)
    assert rel(gj, rj) <= GRAD_REL and rel(gk, rk) <= GRAD_REL, (rel(gj, rj), rel(gk, rk))


def test_autograd_function_and_zero_cases(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300.autograd import render
    p = inputs.random_small(130, shape=(10, 9, 12), n_freq=2, n_src=2, num_rays=80, horizon=8.0)
    j = torch.from_numpy(p.j).cuda().requires_grad_(True)
    k = torch.from_numpy(p.kappa).cuda().requires_grad_(True)
    s = torch.from_numpy(p.sources).cuda()
    F = render(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
    W = torch.randn_like(F)
    (F * W).sum().backward()
    rj, rk = oracle_backward(p, W.cpu().numpy().astype(np.float64))
    assert rel(j.grad.cpu().numpy(), rj) <= GRAD_REL and rel(k.grad.cpu().numpy(), rk) <= GRAD_REL
    # 3-D (one bin) inputs, gradient only for j
    j1 = torch.from_numpy(p.j[0]).cuda().requires_grad_(True)
    F1 = render(j1, torch.from_numpy(p.kappa[0]).cuda(), s, p.num_rays, p.step_size, 1.0, p.time_step)
    assert F1.shape == j1.shape
    F1.sum().backward()
    assert j1.grad.shape == j1.shape and torch.isfinite(j1.grad).all()
    # no sources: zero gradients
    from paper_2511_09389_gb300.api import Grid
    g = Grid(p.shape, 8)
    gj, gk = g.backward(torch.ones_like(j), j.detach(), k.detach(), s[:0], p.num_rays, p.step_size, 1.0,
                        p.time_step)
    assert torch.count_nonzero(gj).item() == 0 and torch.count_nonzero(gk).item() == 0


def test_amplitude_inversion_on_gpu(torch_cuda):
    """Sec. 4: recover a scalar amplitude A of a fixed template e0 from a reference field by
    gradient descent through the differentiable march; the answer is the closed-form MSE
    minimiser <F0, I_ref> / <F0, F0> (F is linear in j)."""
    torch = torch_cuda
    from paper_2511_09389_gb300.autograd import render
    p = inputs.single_source_uniform(n=24, num_rays=768, horizon=10.0)
    e0 = torch.from_numpy(p.j).cuda()
    k = torch.from_numpy(p.kappa).cuda()
    s = torch.from_numpy(p.sources).cuda()
    F0 = render(e0, k, s, p.num_rays, p.step_size, 1.0, p.time_step).double()
    gen = torch.Generator(device="cuda").manual_seed(0)
    Iref = 2.7 * F0 * (1 + 0.05 * torch.randn(F0.shape, generator=gen, device="cuda", dtype=torch.float64))
    A_star = (F0 * Iref).sum() / (F0 * F0).sum()
    curv = 2 * (F0 * F0).sum()
    A = torch.zeros((), device="cuda", dtype=torch.float32, requires_grad=True)
    for _ in range(25):
        F = render(A * e0, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
        loss = ((F.double() - Iref) ** 2).sum()
        A.grad = None
        loss.backward()
        with torch.no_grad():
            A -= (0.8 * A.grad.double() / curv).float()
    assert abs(A.item() - A_star.item()) <= 1e-4 * abs(A_star.item()), (A.item(), A_star.item())


# ---- gradients with respect to the source positions and parameters built into j / kappa ----

def gpu_backward_sources(torch, p, G, **opts):
    from paper_2511_09389_gb300.api import Grid
    g = Grid(p.shape, 8, **opts)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    gj, gk, gs = g.backward(t(G), t(p.j), t(p.kappa), t(p.sources), p.num_rays, p.step_size,
                            p.radiation_velocity, p.time_step, need_sources=True)
    torch.cuda.synchronize()
    return gj.cpu().numpy(), gk.cpu().numpy(), gs.cpu().numpy()


@pytest.mark.parametrize("n_freq,stride", [(1, 4), (1, 16), (2, 8), (3, 32), (4, 4), (5, 16)])
def test_source_gradient_matches_oracle(torch_cuda, n_freq, stride):
    p = inputs.random_small(200 + n_freq, shape=(14, 11, 17), n_freq=n_freq, n_src=4, num_rays=97,
                            step_size=0.6, horizon=15.0)
    G = np.random.default_rng(7 + n_freq).standard_normal(p.j.shape)
    gj, gk, gs = gpu_backward_sources(torch_cuda, p, G, ckpt_stride=stride)
    ns = oracle.num_substeps(p.step_size, p.radiation_velocity, p.time_step)
    rs = oracle.source_gradient(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns, G)
    assert rel(gs, rs) <= GRAD_REL, rel(gs, rs)
    # the field gradients of the same call are those of rt_backward
    rj, rk = oracle_backward(p, G)
    for b in range(n_freq):
        assert rel(gj[b], rj[b]) <= GRAD_REL and rel(gk[b], rk[b]) <= GRAD_REL


def test_source_gradient_full_size_inverse_workload(torch_cuda):
    """64^3 lognormal kappa, 8 sources, N_Omega 3072, N_s 128, G = the log-field loss gradient
    shape (a random field), against the oracle."""
    p = inputs.inverse_problem()
    G = np.random.default_rng(11).standard_normal(p.j.shape)
    _, _, gs = gpu_backward_sources(torch_cuda, p, G)
    ns = oracle.num_substeps(p.step_size, p.radiation_velocity, p.time_step)
    rs = oracle.source_gradient(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns, G)
    assert rel(gs, rs) <= GRAD_REL, rel(gs, rs)


def test_autograd_sources_kappa_scale_and_amplitudes(torch_cuda):
    """Parameters of the kind Sec. 4 names: a global kappa scale, per-source amplitudes (j as a
    sum of per-source templates), and the source positions; gradients through RTFunction
    against the oracle's adjoint composed by hand."""
    torch = torch_cuda
    from paper_2511_09389_gb300.autograd import render
    rng = np.random.default_rng(3)
    shape = (16, 14, 18)
    centres = np.array([[5.2, 6.7, 8.1], [10.4, 7.3, 9.9], [7.7, 4.2, 12.5]])
    templ = np.stack([inputs.gaussian_blobs(shape, c[None], 1.5, 1.0) for c in centres]).astype(np.float64)
    kap0 = (0.03 + 0.05 * rng.random(shape))
    amps = np.array([1.0, 0.6, 1.7])
    alpha = 1.3
    G = rng.standard_normal((2,) + shape)
    num_rays, ds, dt = 256, 0.5, 9.0
    nus = np.array([1.0, 1.5])

    A = torch.tensor(amps, dtype=torch.float32, device="cuda", requires_grad=True)
    al = torch.tensor(alpha, dtype=torch.float32, device="cuda", requires_grad=True)
    S = torch.tensor(centres, dtype=torch.float32, device="cuda", requires_grad=True)
    T = torch.from_numpy(templ.astype(np.float32)).cuda()
    K0 = torch.from_numpy(kap0.astype(np.float32)).cuda()
    nu = torch.from_numpy(nus.astype(np.float32)).cuda()
    j = torch.einsum("i,ixyz->xyz", A, T)[None].expand(2, *shape).contiguous()
    kappa = al * K0[None] * nu[:, None, None, None] ** -3.0
    F = render(j, kappa, S, num_rays, ds, 1.0, dt)
    (F * torch.from_numpy(G.astype(np.float32)).cuda()).sum().backward()

    jn = np.einsum("i,ixyz->xyz", amps, templ)[None].repeat(2, axis=0)
    kn = alpha * kap0[None] * nus[:, None, None, None] ** -3.0
    ns = oracle.num_substeps(ds, 1.0, dt)
    rj, rk = oracle.backward(jn, kn, centres, num_rays, ds, ns, G)
    dA = np.einsum("bxyz,ixyz->i", rj, templ)
    dal = float((rk * kn / alpha).sum())
    dS = oracle.source_gradient(jn, kn, centres, num_rays, ds, ns, G)
    assert rel(A.grad.cpu().numpy(), dA) <= GRAD_REL
    assert abs(al.grad.item() - dal) <= GRAD_REL * abs(dal)
    assert rel(S.grad.cpu().numpy(), dS) <= GRAD_REL


@pytest.mark.parametrize("n_freq,stride,plan", [(1, 16, None), (3, 8, None), (5, 32, (4, 64, 0, 2, 1)), (2, 16, None),
                                                 (1, 16, (1, 32, 0, 2)), (2, 8, (2, 64, 0, 2)), (4, 8, (4, 32, 4, 1)),
                                                 (3, 16, (4, 64, 4, 2)), (2, 4, (2, 32, 4, 2)), (2, 8, (2, 32, 4, 1))])
def test_recorded_checkpoints_give_the_same_gradients(torch_cuda, n_freq, stride, plan):
    """record_checkpoints: the forward march stores the reverse march's checkpoints and the
    adjoint skips its forward sweep; gradients as without it. A backward whose arguments
    differ from the recorded call (another j buffer) makes its own sweep."""
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.random_small(300 + n_freq, shape=(14, 11, 17), n_freq=n_freq, n_src=4, num_rays=97,
                            step_size=0.6, horizon=15.0)
    G = np.random.default_rng(n_freq).standard_normal(p.j.shape)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    j, k, s, Gt = t(p.j), t(p.kappa), t(p.sources), t(G)
    g = Grid(p.shape, 8, ckpt_stride=stride, record_checkpoints=True, plan=plan)
    F = g.advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step).cpu().numpy()
    if plan is not None and plan[2] == 4:   # recorded with the gathers a substep ahead
        assert g.last_plan()["prefetch"] == 4 and g.last_plan()["lanes_per_ray"] == plan[3]
    gj, gk, gs = g.backward(Gt, j, k, s, p.num_rays, p.step_size, 1.0, p.time_step, need_sources=True)
    rj, rk = oracle_backward(p, G)
    ns = oracle.num_substeps(p.step_size, p.radiation_velocity, p.time_step)
    rs = oracle.source_gradient(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns, G)
    gj, gk, gs = gj.cpu().numpy(), gk.cpu().numpy(), gs.cpu().numpy()
    for b in range(n_freq):
        assert rel(gj[b], rj[b]) <= GRAD_REL and rel(gk[b], rk[b]) <= GRAD_REL
    assert rel(gs, rs) <= GRAD_REL
    # the forward field is the plain advance's
    R = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns)
    for b in range(n_freq):
        assert np.linalg.norm(F[b] - R[b]) <= 1e-5 * np.linalg.norm(R[b])
    # a different j buffer (same values): no reuse, same gradients
    j2 = j.clone()
    gj2, gk2 = g.backward(Gt, j2, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
    assert rel(gj2.cpu().numpy(), rj) <= GRAD_REL and rel(gk2.cpu().numpy(), rk) <= GRAD_REL
    # then the original call again: its recording was replaced by that sweep, still correct
    gj3, _ = g.backward(Gt, j, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
    assert rel(gj3.cpu().numpy(), rj) <= GRAD_REL


@pytest.mark.parametrize("n_freq,which", [(1, "j"), (1, "kappa"), (4, "j"), (3, "sources")])
def test_recorded_checkpoints_after_inputs_rewritten_in_place(torch_cuda, n_freq, which):
    """A C caller that rewrites j_map, kappa_map or source_pos IN PLACE between a recording
    rt_advance and rt_backward (same pointers, same scalars) gets the gradients of the new
    contents: the reverse march compares a content hash of the inputs taken at the forward with
    one taken at the backward, on the device, and repeats the forward sweep when they differ. The
    result matches a handle that never recorded (up to the order of the FP32 gradient atomics), and
    both match the oracle's adjoint of the new inputs; with the inputs untouched the recording is
    used and gives the same gradients within the bar."""
    import ctypes
    torch = torch_cuda
    from paper_2511_09389_gb300 import _native
    from paper_2511_09389_gb300.api import Grid
    lib = _native.load()
    p = inputs.random_small(340 + n_freq, shape=(13, 12, 15), n_freq=n_freq, n_src=3, num_rays=90,
                            step_size=0.6, horizon=14.0)
    G = np.random.default_rng(9).standard_normal(p.j.shape)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    j, k, s, Gt = t(p.j), t(p.kappa), t(p.sources), t(G)
    out = torch.empty_like(j)
    gj, gk, gsrc = torch.empty_like(j), torch.empty_like(j), torch.empty_like(s)
    g = Grid(p.shape, 8, record_checkpoints=True)
    stream = torch.cuda.current_stream().cuda_stream

    def advance():
        _native.check(lib.rt_advance(g._h, j.data_ptr(), k.data_ptr(), s.data_ptr(), s.shape[0], p.num_rays,
                                     ctypes.c_float(p.step_size), ctypes.c_float(1.0), ctypes.c_float(p.time_step),
                                     n_freq, out.data_ptr(), 0, stream))

    def backward(h):
        _native.check(lib.rt_backward_sources(h, Gt.data_ptr(), j.data_ptr(), k.data_ptr(), s.data_ptr(), s.shape[0],
                                              p.num_rays, ctypes.c_float(p.step_size), ctypes.c_float(1.0),
                                              ctypes.c_float(p.time_step), n_freq, gj.data_ptr(), gk.data_ptr(),
                                              gsrc.data_ptr(), stream))
        torch.cuda.synchronize()
        return gj.cpu().numpy().copy(), gk.cpu().numpy().copy(), gsrc.cpu().numpy().copy()

    advance()
    kept = backward(g._h)                       # untouched inputs: the recording is reused
    rj, rk = oracle_backward(p, G)
    assert rel(kept[0], rj) <= GRAD_REL and rel(kept[1], rk) <= GRAD_REL

    advance()                                   # record again, then rewrite in place
    if which == "j":
        j.mul_(1.7).add_(0.01)
    elif which == "kappa":
        k.mul_(1.3)
    else:
        s[0, 1] += 0.37
    torch.cuda.synchronize()
    new = backward(g._h)
    fresh = Grid(p.shape, 8)                    # never recorded: its own forward sweep
    ref = backward(fresh._h)
    for a, b in zip(new, ref):
        assert rel(a, b) <= 1e-5     # stale checkpoints would be off by the rewrite itself
    q = inputs.Problem(p.name, j.cpu().numpy(), k.cpu().numpy(), s.cpu().numpy(), p.num_rays, p.step_size,
                       p.radiation_velocity, p.time_step)
    nj, nk = oracle_backward(q, G)
    assert rel(new[0], nj) <= GRAD_REL and rel(new[1], nk) <= GRAD_REL
    g.close()
    fresh.close()


def test_checkpoint_stride_autotuned_and_reused(torch_cuda):
    """With autotune and an automatic stride, the first backward of a shape class times the
    reverse march for K in {4, 8, 16, 32} and keeps the fastest; gradients at the chosen K match
    the oracle; the next recording forward records with it and the backward reuses it."""
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.random_small(360, shape=(16, 14, 18), n_freq=1, n_src=3, num_rays=120, step_size=0.5, horizon=16.0)
    G = np.random.default_rng(3).standard_normal(p.j.shape)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    j, k, s, Gt = t(p.j), t(p.kappa), t(p.sources), t(G)
    g = Grid(p.shape, 1, autotune=True, record_checkpoints=True)
    g.advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
    gj, gk = g.backward(Gt, j, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
    info = g.last_ckpt_stride()
    assert info["stride"] in (4, 8, 16, 32) and info["tuned_ms"] > 0
    rj, rk = oracle_backward(p, G)
    assert rel(gj.cpu().numpy(), rj) <= GRAD_REL and rel(gk.cpu().numpy(), rk) <= GRAD_REL
    g.advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
    gj2, gk2 = g.backward(Gt, j, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
    assert g.last_ckpt_stride() == info
    assert rel(gj2.cpu().numpy(), rj) <= GRAD_REL and rel(gk2.cpu().numpy(), rk) <= GRAD_REL
    for K in (4, 8):   # the new strides against the oracle too
        gK = Grid(p.shape, 1, ckpt_stride=K, record_checkpoints=True)
        gK.advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
        a, b = gK.backward(Gt, j, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
        assert gK.last_ckpt_stride()["stride"] == K
        assert rel(a.cpu().numpy(), rj) <= GRAD_REL and rel(b.cpu().numpy(), rk) <= GRAD_REL


def test_emissivity_inversion_reduced_size(torch_cuda):
    """Config-4 inversion at reduced size: j recovered from zero by Adam (projected onto j >= 0) on
    the MSE of the log field through the differentiable march, with the checkpoint stride tuned.
    The loss falls and the recovered emissivity correlates with the target blobs."""
    torch = torch_cuda
    from paper_2511_09389_gb300 import inversion
    from paper_2511_09389_gb300.api import Grid
    p = inputs.inverse_problem(n=32, n_blobs=4, num_rays=768, horizon=32.0, seed=4100)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    j_true, k, s = t(p.j), t(p.kappa), t(p.sources)
    g = Grid(p.shape, 1, record_checkpoints=True, autotune=True)
    target = g.advance(j_true, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
    res = inversion.recover_emissivity(target, k, s, p.num_rays, p.step_size, 1.0, p.time_step, iterations=80,
                                       lr=5e-2, grid=g)
    L = res["losses"]
    corr = inversion.correlation(res["j"], j_true)
    print(f"inversion 32^3: loss {L[0]:.3e} -> {L[-1]:.3e}, correlation {corr:.3f}, K {res['ckpt_stride']}")
    assert L[-1] < 0.05 * L[0]
    assert corr > 0.5          # FP64 oracle, same settings: loss x 7e-3, correlation 0.74
    assert float(res["j"].min()) >= 0.0


@pytest.mark.parametrize("n_freq,record", [(1, True), (2, False)])
def test_native_inversion_loop_matches_autograd_loop(torch_cuda, n_freq, record):
    """rt_invert_emissivity (the loop in the library: recording forward, fused log misfit and its
    gradient, reverse march, Adam with the projection fused) against the same iterations written
    with torch autograd: RTFunction for the march, the loss in torch ops, rt_adam_step, clamp.
    Both sum their deposits with FP32 atomics in run-dependent order, so losses and the recovered
    j agree to rounding-level tolerances, not bitwise. Also: the loss history has iterations + 1
    entries, j stays >= 0, and zero iterations return the start's loss and leave j unchanged. Two
    bins: one loss over both; without recorded checkpoints every reverse march runs its own
    forward sweep."""
    torch = torch_cuda
    from paper_2511_09389_gb300 import inversion
    from paper_2511_09389_gb300.api import Grid, adam_step
    from paper_2511_09389_gb300.autograd import RTFunction
    p = inputs.inverse_problem(n=24, n_blobs=3, num_rays=512, horizon=24.0, seed=4200)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    j_true, k, s = t(p.j), t(p.kappa), t(p.sources)
    if n_freq == 2:   # a second bin with more opaque kappa and a dimmer emissivity
        j_true = torch.cat([j_true, 0.5 * j_true])
        k = torch.cat([k, 1.8 * k])
    g = Grid(p.shape, n_freq, record_checkpoints=record)
    target = g.advance(j_true, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
    iters, lr, eps_rel = 25, 5e-2, 1e-2
    res = inversion.recover_emissivity(target, k, s, p.num_rays, p.step_size, 1.0, p.time_step, iterations=iters,
                                       lr=lr, eps_rel=eps_rel, grid=g)
    # the same loop in torch
    eps = eps_rel * float(target.max())
    log_t = torch.log(target + eps)
    j = torch.zeros_like(k)
    m, v = torch.zeros_like(j), torch.zeros_like(j)
    ref_losses = []
    for it in range(1, iters + 1):
        jv = j.detach().requires_grad_(True)
        F = RTFunction.apply(jv, k, s, p.num_rays, p.step_size, 1.0, p.time_step, g)
        loss = inversion.log_field_loss(F, log_t, eps)
        loss.backward()
        ref_losses.append(float(loss.detach()))
        adam_step(j, jv.grad, m, v, lr=lr, step=it)
        j.clamp_(min=0.0)
    L = np.array(res["losses"])
    assert L.shape == (iters + 1,)
    rel_loss = np.abs(L[:iters] - ref_losses) / np.array(ref_losses)
    rel_j = float((res["j"] - j).norm() / j.norm())
    print(f"native vs autograd loop: max loss rel diff {rel_loss.max():.2e}, j rel-L2 {rel_j:.2e}, "
          f"loss {L[0]:.3e} -> {L[-1]:.3e}")
    assert rel_loss.max() < 1e-3 and rel_j < 1e-2
    assert float(res["j"].min()) >= 0.0 and L[-1] < L[0]
    res0 = inversion.recover_emissivity(target, k, s, p.num_rays, p.step_size, 1.0, p.time_step, iterations=0,
                                        grid=g, j0=j)
    F = g.advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
    assert len(res0["losses"]) == 1 and torch.equal(res0["j"], j)
    assert abs(res0["losses"][0] - float(inversion.log_field_loss(F, log_t, eps))) <= 1e-5 * res0["losses"][0]


def test_native_inversion_rejects_bad_arguments(torch_cuda):
    """Scalars, NULL arrays, n_freq, aliasing and overlapping loss buffers are refused with
    RT_ERR_INVALID_ARG before anything is enqueued (j is left as it was)."""
    torch = torch_cuda
    from paper_2511_09389_gb300 import _native
    from paper_2511_09389_gb300.api import Grid
    lib = _native.load()
    g = Grid((8, 8, 8), 1)
    z = lambda: torch.rand(1, 8, 8, 8, device="cuda")
    tgt, kap, jm = z(), z(), z()
    j0 = jm.clone()
    src = torch.full((1, 3), 3.5, device="cuda")
    losses = torch.zeros(8, device="cuda")
    P = lambda t: t.data_ptr() if t is not None else None
    cases = [dict(tgt=None), dict(iters=-1), dict(lr=0.0), dict(lr=float("nan")), dict(eps_rel=0.0),
             dict(eps_rel=float("inf")), dict(nf=2), dict(jm=tgt), dict(jm=kap), dict(losses=jm), dict(losses=None)]
    for c in cases:
        a = dict(tgt=tgt, kap=kap, nf=1, iters=3, lr=1e-2, eps_rel=1e-2, jm=jm, losses=losses)
        a.update(c)
        st = lib.rt_invert_emissivity(g._h, P(a["tgt"]), P(a["kap"]), P(src), 1, 16, 0.5, 1.0, 2.0, a["nf"], a["iters"],
                                      a["lr"], a["eps_rel"], P(a["jm"]), P(a["losses"]), None)
        assert st == 1, c
    torch.cuda.synchronize()
    assert torch.equal(jm, j0)
