"""GPU parity of the forward march (rt_advance) against the FP64 oracle.

Bar (FP32 path vs FP64 oracle): per bin, relative L2 error <= 1e-5 and max-abs error
<= 1e-4 * max|F_oracle| (the pointwise relative error is undefined past the light-travel
horizon, where the field is zero). Cell indices and the direction lattice are bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2511_09389_gb300 import inputs

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
MAX_ABS_REL = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2511_09389_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


def errors(F, R):
    """Per-bin (relative L2, max-abs relative to max|R|)."""
    F = np.asarray(F, np.float64).reshape(R.shape)
    out = []
    for b in range(R.shape[0]):
        d = F[b] - R[b]
        nr = np.linalg.norm(R[b])
        mx = np.abs(R[b]).max()
        out.append((np.linalg.norm(d) / nr if nr > 0 else np.linalg.norm(d),
                    np.abs(d).max() / mx if mx > 0 else np.abs(d).max()))
    return out


def assert_parity(F, R, rel=REL_L2, mx=MAX_ABS_REL):
    for b, (e2, emax) in enumerate(errors(F, R)):
        assert e2 <= rel and emax <= mx, f"bin {b}: rel-L2 {e2:.3e}, max-abs-rel {emax:.3e}"


def run_gpu(torch, p, ns=None, kappa_mode=0, grid=None, **kw):
    from paper_2511_09389_gb300.api import Grid
    g = grid or Grid(p.shape, max(8, p.n_freq), kappa_mode=kappa_mode)
    j = torch.from_numpy(p.j).cuda()
    k = torch.from_numpy(p.kappa).cuda()
    s = torch.from_numpy(p.sources).cuda()
    dt = p.time_step if ns is None else ns * p.step_size
    out = g.advance(j, k, s, p.num_rays, p.step_size, p.radiation_velocity, dt, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def run_oracle(p, ns=None, kappa_mode=0, ray_range=None):
    if ns is None:
        ns = oracle.num_substeps(p.step_size, p.radiation_velocity, p.time_step)
    return oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns, geom_mode=0,
                          kappa_mode=kappa_mode, ray_range=ray_range)


def test_single_source_uniform_32cubed(torch_cuda):
    """32^3, kappa 0.1, sigma-1 blob at the centre, N_Omega 768, ds 0.5, c dt 16, one bin."""
    p = inputs.single_source_uniform()
    assert_parity(run_gpu(torch_cuda, p), run_oracle(p))


@pytest.mark.parametrize("n_freq", [1, 2, 3, 4, 5, 8])
def test_random_irregular_grids_all_bin_widths(torch_cuda, n_freq):
    """Non-cubic grid, sources outside the box, ragged ray count, every bin-group width."""
    p = inputs.random_small(10 + n_freq, shape=(13, 9, 17), n_freq=n_freq, n_src=5, num_rays=131,
                            step_size=0.6, horizon=14.0)
    assert_parity(run_gpu(torch_cuda, p), run_oracle(p))


@pytest.mark.parametrize("kappa_mode", [0, 1])
def test_kappa_modes(torch_cuda, kappa_mode):
    p = inputs.random_small(21, shape=(16, 12, 10), n_freq=4, n_src=3, num_rays=200, horizon=12.0)
    assert_parity(run_gpu(torch_cuda, p, kappa_mode=kappa_mode), run_oracle(p, kappa_mode=kappa_mode))


def test_cell_trace_bit_exact(torch_cuda):
    from paper_2511_09389_gb300.api import Grid
    shape = (23, 19, 29)
    rng = np.random.default_rng(2)
    for kappa_mode in (0, 1):
        g = Grid(shape, 1, kappa_mode=kappa_mode)
        z = np.zeros((1,) + shape)
        for trial in range(12):
            src = rng.uniform(-3, 25, 3).astype(np.float32)
            nr = int(rng.choice([1, 7, 768, 3072, 12288]))
            ray = int(rng.integers(0, nr))
            ds = float(np.float32(rng.choice([0.5, 0.37, 1.0, 0.125])))
            ns = 200
            b_o, n_o, _ = oracle.trace_ray(z, z, src, nr, ray, ds, ns, geom_mode=0, kappa_mode=kappa_mode)
            b_g, n_g = g.trace_cells(src, nr, ray, ds, ns)
            assert np.array_equal(b_o, b_g) and np.array_equal(n_o, n_g), (kappa_mode, trial)


def test_turbulent_reduced(torch_cuda):
    """Turbulent medium at reduced size: 48^3 lognormal, 6 sources, 4 bins, N_Omega 768,
    N_s 96 (rays cross the box and deposit on its faces)."""
    p = inputs.turbulent(n=48, n_src=6, num_rays=768, horizon=48.0, seed=77)
    assert_parity(run_gpu(torch_cuda, p), run_oracle(p))


@pytest.mark.slow
def test_turbulent_full_size(torch_cuda):
    """The benchmark workload at full size, in the launch configuration the benchmark times:
    128^3, 16 sources, N_Omega 3072, N_s 256, 4 bins (the oracle takes a few seconds per
    bin on one core)."""
    p = inputs.turbulent()
    assert_parity(run_gpu(torch_cuda, p), run_oracle(p))


def test_uniform_closed_form_on_gpu(torch_cuda):
    """Uniform j0, kappa: sum over cells = n_src * 4 pi sum_k (k+1) j0 ds exp(-kappa k ds)."""
    n, ns, ds, j0, kap = 40, 77, 0.5, 0.8, 0.05
    p = inputs.Problem("u", np.full((2, n, n, n), j0, np.float32),
                       np.stack([np.full((n, n, n), kap, np.float32), np.zeros((n, n, n), np.float32)]),
                       np.array([[3.0, 20.0, 38.5], [-4.0, 10.0, 10.0]], np.float32), 1000, ds, 1.0, ns * ds)
    F = run_gpu(torch_cuda, p)
    k = np.arange(ns)
    for b, kb in enumerate((kap, 0.0)):
        expect = 2 * 4 * math.pi * np.sum((k + 1) * j0 * ds * np.exp(-kb * k * ds))
        assert abs(F[b].sum(dtype=np.float64) / expect - 1) < 2e-5


def test_shards_accumulate_and_empty_cases(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.random_small(31, shape=(12, 12, 12), n_freq=3, n_src=4, num_rays=300, horizon=10.0)
    g = Grid(p.shape, 8)
    j, k, s = (torch.from_numpy(a).cuda() for a in (p.j, p.kappa, p.sources))
    full = g.advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
    acc = torch.zeros_like(full)
    for rb, re in [(0, 1), (1, 100), (100, 100), (100, 300)]:
        g.advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step, out=acc, accumulate=True, ray_range=(rb, re))
    assert torch.allclose(acc, full, rtol=1e-5, atol=1e-6 * full.abs().max().item())
    # accumulate adds to what is there
    twice = g.advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step, out=full.clone(), accumulate=True)
    assert torch.allclose(twice, 2 * full, rtol=1e-5, atol=1e-6 * full.abs().max().item())
    # no sources, zero horizon: zero field (overwriting garbage)
    junk = torch.full_like(full, 7.0)
    g.advance(j, k, s[:0], p.num_rays, p.step_size, 1.0, p.time_step, out=junk)
    assert torch.count_nonzero(junk).item() == 0
    junk.fill_(7.0)
    g.advance(j, k, s, p.num_rays, p.step_size, 1.0, 0.0, out=junk)
    assert torch.count_nonzero(junk).item() == 0
    torch.cuda.synchronize()


def test_host_entry_point_matches_device(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.random_small(41, shape=(20, 18, 16), n_freq=4, n_src=3, num_rays=256, horizon=16.0)
    g = Grid(p.shape, 8)
    dev = g.advance(*(torch.from_numpy(a).cuda() for a in (p.j, p.kappa, p.sources)), p.num_rays,
                    p.step_size, 1.0, p.time_step).cpu().numpy()
    host = g.advance_host(p.j, p.kappa, p.sources, p.num_rays, p.step_size, 1.0, p.time_step)
    np.testing.assert_allclose(host, dev, rtol=2e-5, atol=1e-6 * np.abs(dev).max())
    assert_parity(host, run_oracle(p))


def test_invalid_arguments_raise(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid, RTError
    g = Grid((8, 8, 8), 2)
    j = torch.ones(2, 8, 8, 8, device="cuda")
    s = torch.zeros(1, 3, device="cuda")
    bad = [dict(num_rays=0), dict(step_size=0.0), dict(step_size=-1.0), dict(radiation_velocity=0.0),
           dict(time_step=-1.0), dict(ray_range=(5, 2)), dict(ray_range=(0, 11))]
    for b in bad:
        kw = dict(num_rays=10, step_size=0.5, radiation_velocity=1.0, time_step=2.0)
        kw.update(b)
        with pytest.raises(RTError, match="INVALID_ARG"):
            g.advance(j, j, s, **kw)
    with pytest.raises(RTError, match="INVALID_ARG"):
        Grid((8, 8, 8), 1).advance(j, j, s, 10, 0.5, 1.0, 2.0)      # n_freq above max_freq
    with pytest.raises(RTError, match="INVALID_ARG"):
        g.advance(j, j, s, 10, 0.5, 1.0, 2.0, out=j)                  # out aliases an input


def test_deterministic_mode_parity_and_bitwise_reproducible(torch_cuda):
    """Fixed-point accumulation: the field meets the same bar against the oracle and is bitwise
    identical across runs and across launch plans (bins per thread, block size, corner slots
    gathered in time or a substep ahead), i.e. for any order in which the deposits arrive."""
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.random_small(51, shape=(20, 16, 24), n_freq=5, n_src=4, num_rays=300, horizon=18.0)
    j, k, s = (torch.from_numpy(a).cuda() for a in (p.j, p.kappa, p.sources))
    outs = []
    for plan in [(4, 32, 0), (4, 32, 0), (1, 64, 0), (2, 128, 0), (4, 256, 0), (4, 32, 4), (1, 64, 4), (2, 32, 4)]:
        g = Grid(p.shape, 8, deterministic=True, plan=plan)
        outs.append(g.advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step).cpu().numpy())
        g.close()
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32))
    assert_parity(outs[0], run_oracle(p))


def test_deterministic_mode_full_size(torch_cuda):
    """The benchmark workload in deterministic mode: 128^3, 16 sources, N_Omega 3072, N_s 256,
    4 bins -- parity with the oracle and run-to-run bit equality."""
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid
    p = inputs.turbulent()
    g = Grid(p.shape, 8, deterministic=True)
    j, k, s = (torch.from_numpy(a).cuda() for a in (p.j, p.kappa, p.sources))
    a = g.advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step).cpu().numpy()
    b = g.advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step).cpu().numpy()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert_parity(a, run_oracle(p))


@pytest.mark.parametrize("plan", [(4, 64, 0, 2), (1, 128, 0, 2), (2, 32, 0, 2), (4, 32, 0, 2), (4, 256, 1, 1), (2, 64, 1, 1), (4, 32, 2, 1), (1, 64, 2, 1),
                                  (1, 32, 0, 1), (4, 32, 0, 1, 1), (2, 128, 1, 1, 1), (1, 64, 1, 1, 1),
                                  (1, 32, 2, 1, 1), (1, 256, 0, 1, 1), (1, 64, 1, 1, 0), (4, 32, 3, 1),
                                  (2, 64, 3, 1, 0), (1, 64, 3, 1, 1), (4, 64, 3, 1, 1),
                                  (4, 32, 4, 1), (2, 64, 4, 1), (1, 128, 4, 1),
                                  (4, 64, 4, 2), (4, 32, 4, 2), (2, 32, 4, 2), (1, 128, 4, 2)])
def test_every_launch_plan_meets_parity(torch_cuda, plan):
    """Each launch plan the autotuner may pick (bins per group, block, prefetch, lanes per ray,
    source deposit tiles) on a ragged multi-bin problem."""
    p = inputs.random_small(60, shape=(18, 14, 22), n_freq=6, n_src=3, num_rays=257, horizon=16.0)
    from paper_2511_09389_gb300.api import Grid
    g = Grid(p.shape, 8, plan=plan)
    assert_parity(run_gpu(torch_cuda, p, grid=g), run_oracle(p))


@pytest.mark.parametrize("plan", [(1, 32, 1, 1, 1), (1, 128, 0, 1, 1), (4, 64, 0, 1, 1), (2, 32, 2, 1, 1),
                                  (1, 64, 3, 1, 1), (4, 32, 3, 1, 1)])
def test_source_tiles_with_clustered_and_face_sources(torch_cuda, plan):
    """Source deposit tiles: many sources packed into a few cells (the tiles overlap and take
    most deposits), plus sources on and outside the faces and corners (the tile origin is moved
    inside the grid; rays that start outside it never use it). Every bin against the oracle."""
    from paper_2511_09389_gb300.api import Grid
    rng = np.random.Generator(np.random.PCG64(77))
    shape = (16, 12, 20)
    nf = plan[0] + 1 if plan[0] > 1 else 1
    j = rng.uniform(0.0, 1.0, size=(nf,) + shape).astype(np.float32)
    kap = rng.uniform(0.0, 0.3, size=(nf,) + shape).astype(np.float32)
    cluster = np.array([7.0, 5.0, 9.0]) + rng.uniform(-1.2, 1.2, size=(10, 3))
    faces = np.array([[0.0, 0.0, 0.0], [15.0, 11.0, 19.0], [-2.0, 5.5, 9.0], [16.5, -0.7, 21.0], [3.0, 11.0, 0.25]])
    src = np.concatenate([cluster, faces]).astype(np.float32)
    p = inputs.Problem("tiles", j, kap, src, 300, 0.5, 1.0, 10.0)
    g = Grid(p.shape, 8, plan=plan)
    F = run_gpu(torch_cuda, p, grid=g)
    assert g.last_plan()["tile"] == 1
    assert_parity(F, run_oracle(p))


@pytest.mark.parametrize("step_size", [0.13, 0.5, 1.0, 1.7, 3.2])
@pytest.mark.parametrize("plan", [(4, 32, 0), (1, 64, 0, 1, 1), (2, 32, 0, 1, 0), (4, 64, 3), (4, 32, 0, 2), (1, 64, 0, 2),
                                  (4, 32, 4), (1, 64, 4, 1), (2, 32, 4), (4, 32, 4, 2), (1, 64, 4, 2)])
def test_corner_slots_across_step_sizes(torch_cuda, plan, step_size):
    """Gathers mode 0 keeps a face shared by consecutive corner sets (a step of one cell along an
    axis) and flushes everything else. Steps much shorter than a cell (long runs in one set), of
    exactly one cell, and of more than one cell (no shared face: every corner leaves), with sources
    inside, on and outside the faces (clamped pairs that collapse and reopen), on a box with one
    axis of a single cell, against the oracle."""
    from paper_2511_09389_gb300.api import Grid
    for shape in ((14, 11, 17), (9, 1, 12)):
        p = inputs.random_small(90, shape=shape, n_freq=5, n_src=4, num_rays=211, step_size=step_size,
                                horizon=14.0)
        g = Grid(p.shape, 8, plan=plan)
        assert_parity(run_gpu(torch_cuda, p, grid=g), run_oracle(p))


@pytest.mark.parametrize("accumulation,plan,n_src,expect", [
    ("auto", None, 40, "fixed"), ("auto", (1, 32, 0, 1), 40, "fixed"), ("auto", (1, 64, 0, 2), 40, "fixed"),
    ("auto", (1, 64, 1, 1), 40, "fixed"), ("auto", (1, 64, 3, 1), 40, "fixed"), ("auto", (1, 64, 1, 1, 1), 40, "fp32"),
    ("auto", (4, 32, 0, 1), 40, "fixed"), ("auto", None, 4, "fp32"), ("auto", (4, 32, 0, 1), 4, "fp32"),
    ("fp32", (1, 64, 0, 2), 40, "fp32"), ("fp32", None, 40, "fp32"), ("fp64", None, 4, "fp64"),
    ("fp64", (1, 32, 0, 1), 4, "fp64"), ("fp64", (4, 32, 0, 1), 4, "fp64"), ("fp64", (2, 64, 0, 1), 4, "fp64"),
    ("fp64", (1, 64, 1, 1, 1), 4, "fp64"), ("fixed", (4, 64, 0, 1), 4, "fixed"), ("fixed", (1, 64, 0, 2), 4, "fixed"),
    ("fixed", (4, 64, 4, 2), 4, "fixed"), ("auto", (1, 64, 4, 2), 40, "fixed"), ("fp32", (4, 32, 4, 2), 40, "fp32")])
def test_accumulation_modes_meet_parity(torch_cuda, accumulation, plan, n_src, expect):
    """rt_options.accumulation on a ragged problem with sources on and outside the faces: FP32, FP64
    and 64-bit fixed-point sums all meet the bar against the oracle. The automatic mode sums in
    FP32 when the call deposits few updates per cell (4 sources here: ~4 per cell and bin) and in
    fixed point when it deposits many (40 sources: ~40), unless a plan pins source tiles (FP32);
    a pinned gathers mode that has no fixed-point kernel falls back to corner slots, and an 8-byte
    accumulation with tiles pinned drops the tiles. The handle reports what it used."""
    from paper_2511_09389_gb300.api import Grid
    nf = 1 if plan is None or plan[0] == 1 else 5
    p = inputs.random_small(61, shape=(17, 13, 21), n_freq=nf, n_src=n_src, num_rays=233, horizon=15.0)
    g = Grid(p.shape, 8, plan=plan, accumulation=accumulation)
    F = run_gpu(torch_cuda, p, grid=g)
    assert g.last_accumulation() == expect
    if expect != "fp32":
        assert g.last_plan()["tile"] == 0
    R = run_oracle(p)
    assert_parity(F, R)
    # accumulate = 1 adds the new field to what out holds
    import torch
    out = torch.from_numpy(F).cuda()
    j, k, s = (torch.from_numpy(a).cuda() for a in (p.j, p.kappa, p.sources))
    g.advance(j, k, s, p.num_rays, p.step_size, p.radiation_velocity, p.time_step, out=out, accumulate=True)
    assert_parity(out.cpu().numpy(), 2.0 * R)
    g.close()


def test_one_bin_sums_on_clustered_sources(torch_cuda):
    """Many sources packed into a few cells: the default one-bin path (fixed-point sums) and FP64
    sums stay at the oracle's values where FP32 sums lose the small deposits the crowded cells take
    (FP32 forced on the same problem is measured beside them, for the record)."""
    from paper_2511_09389_gb300.api import Grid
    rng = np.random.Generator(np.random.PCG64(78))
    shape = (24, 24, 24)
    j = rng.uniform(0.0, 1.0, size=(1,) + shape).astype(np.float32)
    kap = rng.uniform(0.0, 0.2, size=(1,) + shape).astype(np.float32)
    src = (np.array([11.0, 12.0, 11.5]) + rng.uniform(-1.5, 1.5, size=(300, 3))).astype(np.float32)
    p = inputs.Problem("cluster", j, kap, src, 768, 0.5, 1.0, 20.0)
    R = run_oracle(p)
    g = Grid(p.shape, 1)
    F = run_gpu(torch_cuda, p, grid=g)
    assert g.last_accumulation() == "fixed"
    assert_parity(F, R)
    F64 = run_gpu(torch_cuda, p, grid=Grid(p.shape, 1, accumulation="fp64"))
    assert_parity(F64, R)
    F32 = run_gpu(torch_cuda, p, grid=Grid(p.shape, 1, accumulation="fp32"))
    e = [np.linalg.norm(X - R) / np.linalg.norm(R) for X in (F, F64, F32)]
    print(f"300 clustered sources: rel-L2 fixed point {e[0]:.2e}, FP64 {e[1]:.2e}, FP32 {e[2]:.2e}")
    assert max(e[0], e[1]) <= e[2]


@pytest.mark.parametrize("width,shape,step_size", [(1, (17, 13, 21), 0.5), (4, (17, 13, 21), 0.5), (1, (9, 1, 12), 1.7),
                                                   (4, (14, 11, 17), 0.13), (2, (14, 11, 17), 3.2)])
def test_gathers_ahead_sums_equal_corner_slots(torch_cuda, width, shape, step_size):
    """Gathers mode 4 is the corner slots of mode 0 with the entering corners gathered one substep
    early: the same sums flushed at the same points. Summed in fixed point (order-independent),
    the two fields are bitwise equal; and both meet the oracle."""
    from paper_2511_09389_gb300.api import Grid
    nf = 1 if width == 1 else 5
    p = inputs.random_small(95, shape=shape, n_freq=nf, n_src=4, num_rays=199, step_size=step_size, horizon=14.0)
    F = [run_gpu(torch_cuda, p, grid=Grid(p.shape, 8, plan=(width, 32, mode, 1), accumulation="fixed"))
         for mode in (0, 4)]
    assert np.array_equal(F[0].view(np.uint32), F[1].view(np.uint32))
    assert_parity(F[1], run_oracle(p))


@pytest.mark.parametrize("shape,step_size", [((17, 13, 21), 0.5), ((9, 1, 12), 1.7), ((14, 11, 17), 0.13),
                                             ((14, 11, 17), 3.2)])
def test_pair_gathers_ahead_sums_equal_pair_slots(torch_cuda, shape, step_size):
    """Two lanes per ray with gathers mode 4 flush the same per-lane slot sums at the same points
    as two lanes per ray with corner slots (mode 0): one bin summed in fixed point gives bitwise
    equal fields; four bins per lane meet the oracle (short steps, steps over a cell, a box with a
    single-cell axis)."""
    from paper_2511_09389_gb300.api import Grid
    p = inputs.random_small(97, shape=shape, n_freq=1, n_src=4, num_rays=201, step_size=step_size, horizon=14.0)
    F = [run_gpu(torch_cuda, p, grid=Grid(p.shape, 8, plan=(1, 64, mode, 2), accumulation="fixed"))
         for mode in (0, 4)]
    assert np.array_equal(F[0].view(np.uint32), F[1].view(np.uint32))
    assert_parity(F[1], run_oracle(p))
    p = inputs.random_small(98, shape=shape, n_freq=4, n_src=4, num_rays=201, step_size=step_size, horizon=14.0)
    assert_parity(run_gpu(torch_cuda, p, grid=Grid(p.shape, 8, plan=(4, 64, 4, 2), accumulation="fixed")),
                  run_oracle(p))


def test_attenuation_factor_accuracy(torch_cuda):
    """exp(-x) as every march kernel computes it (rt_neg_exp: 2^(-x log2 e)) against FP64 exp:
    the relative error is at most 2^-21 (the base-2 exponential) plus 1.25 |x| 2^-24 wherever
    exp(-x) is a normal FP32 number (x <= 87); beyond that the factor is flushed to zero. The
    second term: the FP32 product y = x log2 e carries the rounding of the product (at most
    |y| 2^-24) and of the constant (FP32 log2 e is off by a relative 1.3e-8 = 0.23 x 2^-24), and
    2^y turns an error e in y into a relative error ln(2) e, with ln(2) log2(e) = 1."""
    torch = torch_cuda
    from paper_2511_09389_gb300 import _native
    lib = _native.load()
    gen = torch.Generator().manual_seed(5)
    x = torch.cat([torch.linspace(0.0, 87.0, 400001, dtype=torch.float64),
                   torch.rand(200000, generator=gen, dtype=torch.float64) * 4.0,
                   torch.tensor([0.0, 1e-30, 1e-7, 0.5, 1.0, 88.0, 100.0, 1e4], dtype=torch.float64)]).float()
    xd = x.cuda()
    yd = torch.empty_like(xd)
    assert lib.rt_neg_exp(xd.data_ptr(), yd.data_ptr(), xd.numel(), None) == 0
    torch.cuda.synchronize()
    y, xx = yd.cpu().double(), x.double()
    ref = torch.exp(-xx)
    normal = xx <= 87.0
    rel = (y[normal] - ref[normal]).abs() / ref[normal]
    bound = 2.0 ** -21 + 1.25 * xx[normal] * 2.0 ** -24
    print(f"neg_exp: max relative error / bound {float((rel / bound).max()):.3f}, "
          f"max relative error {float(rel.max()):.2e}")
    assert bool((rel <= bound).all())
    assert bool((y[xx >= 88.0] == 0).all())
    assert lib.rt_neg_exp(xd.data_ptr(), yd.data_ptr(), -1, None) == 1
