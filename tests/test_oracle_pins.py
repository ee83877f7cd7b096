"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: closed forms of Eq. 2 for
uniform media, the analytic point-source solution (Eq. 3), limits, linearity, a brute-force
double-sum form of the recursion built on scipy's trilinear interpolation, exact identities
of the adjoint, finite differences and the closed-form minimiser of the inversion (Sec. 4).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.ndimage import map_coordinates

import oracle
from paper_2511_09389_gb300 import inputs

# numbers the paper prints, each with its passage (small text fixture)
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_printed_values.json")) as _f:
    PAPER = json.load(_f)

FOUR_PI = 4.0 * math.pi


def _grid_coords(shape):
    return np.stack(np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij"), -1)


# --------------------------------------------------------------------------------------------
# N_s rule (Sec. 2 after Eq. 2; App. A)
# --------------------------------------------------------------------------------------------
def test_num_substeps_rule():
    assert oracle.num_substeps(0.5, 1.0, 16.0) == 32
    assert oracle.num_substeps(0.5, 1.0, 128.0) == 256
    assert oracle.num_substeps(0.5, 1.0, 64.0) == 128
    assert oracle.num_substeps(0.3, 1.0, 0.9) == 3          # 0.9/0.3 is 3.0000000000000004
    assert oracle.num_substeps(0.5, 2.0, 3.1) == 13         # ceil(12.4)
    assert oracle.num_substeps(0.5, 1.0, 0.0) == 0
    assert oracle.num_substeps(0.5, 1.0, 128.0, cap=100) == 100
    with pytest.raises(ValueError):
        oracle.num_substeps(0.0, 1.0, 1.0)


# --------------------------------------------------------------------------------------------
# Fibonacci lattice (Sec. 2)
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 37, 192, 768, 3072, 12288])
def test_fibonacci_lattice(n):
    d = oracle.fibonacci_dirs(n)
    assert d.shape == (n, 3)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, rtol=0, atol=4e-16)
    # z values equally spaced in (-1, 1), first at 1 - 1/n: equal-area bands
    np.testing.assert_allclose(d[:, 2], 1.0 - (2.0 * np.arange(n) + 1.0) / n, rtol=0, atol=1e-15)
    if n >= 3:
        # consecutive azimuths advance by the golden angle pi (3 - sqrt 5) modulo 2 pi
        phi = np.arctan2(d[:, 1], d[:, 0])
        step = np.mod(np.diff(phi), 2 * math.pi)
        np.testing.assert_allclose(step, math.pi * (3 - math.sqrt(5)), atol=1e-9)
    if n >= 192:
        # nearly uniform: the mean direction vanishes
        assert np.linalg.norm(d.mean(0)) < 2.0 / n
    f32 = oracle.fibonacci_dirs_f32(n)
    assert np.array_equal(f32, d.astype(np.float32))


def test_single_direction_is_plus_axis0():
    np.testing.assert_allclose(oracle.fibonacci_dirs(1), [[1.0, 0.0, 0.0]], atol=1e-16)


# --------------------------------------------------------------------------------------------
# Closed forms of Eq. 2 for uniform media (exact identities)
# --------------------------------------------------------------------------------------------
def _uniform_total(j0, kap, ds, ns):
    """Sum over cells of the field for uniform j0, kappa: the recursion gives
    I_{k+1} = (k+1) j0 ds exp(-kappa k ds) on every ray, and the clamped trilinear weights of
    each deposit sum to one, so sum_cells F = 4 pi sum_k (k+1) j0 ds exp(-kappa k ds)."""
    k = np.arange(ns, dtype=np.float64)
    return FOUR_PI * np.sum((k + 1) * j0 * ds * np.exp(-kap * k * ds))


@pytest.mark.parametrize("geom", [0, 1])
@pytest.mark.parametrize("kap", [0.0, 0.07, 0.6])
def test_uniform_medium_closed_form(geom, kap):
    shape = (7, 6, 5)
    ns, ds, j0 = 23, 0.5, 1.7
    # sources inside, on a face and outside the box: clamped deposits keep weight sum one
    src = np.array([[3.2, 2.5, 2.0], [0.0, 5.0, 4.0], [-2.3, 7.1, 1.3]])
    j = np.full((1,) + shape, j0)
    kappa = np.full((1,) + shape, kap)
    F = oracle.advance(j, kappa, src, 41, ds, ns, geom_mode=geom)
    expect = len(src) * _uniform_total(j0, kap, ds, ns)
    np.testing.assert_allclose(F.sum(), expect, rtol=1e-12)
    if kap == 0.0:
        np.testing.assert_allclose(F.sum(), len(src) * FOUR_PI * j0 * ds * ns * (ns + 1) / 2, rtol=1e-12)


def test_zero_emission_gives_zero_field():
    p = inputs.random_small(1)
    F = oracle.advance(np.zeros_like(p.j), p.kappa, p.sources, p.num_rays, p.step_size, 12)
    assert np.all(F == 0.0)


def test_zero_substeps_and_no_sources():
    p = inputs.random_small(2)
    assert np.all(oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, 0) == 0.0)
    assert np.all(oracle.advance(p.j, p.kappa, np.zeros((0, 3)), p.num_rays, p.step_size, 9) == 0.0)


# --------------------------------------------------------------------------------------------
# Worked single-ray example (Eq. 2 by hand, 4 substeps)
# --------------------------------------------------------------------------------------------
def test_single_ray_worked_example():
    """One ray (N_Omega = 1 points along +axis 0) from (1.25, 1.5, 1.75), ds = 0.5, N_s = 4.
    j is affine, j(v) = 1 + v0/2 + v1/4 + v2/8, which trilinear interpolation reproduces
    exactly; kappa = 0.1 + 0.05 v0. Positions x0 = 1.25, 1.75, 2.25, 2.75 sit in cells
    v0 = 1, 1, 2, 2, so kappa_k = 0.15, 0.15, 0.2, 0.2."""
    shape = (6, 6, 6)
    v = _grid_coords(shape)
    j = 1.0 + v[..., 0] / 2 + v[..., 1] / 4 + v[..., 2] / 8
    kap = 0.1 + 0.05 * v[..., 0]
    src = np.array([1.25, 1.5, 1.75])
    ds = 0.5
    xs = [1.25, 1.75, 2.25, 2.75]
    jk = [1.0 + x / 2 + 1.5 / 4 + 1.75 / 8 for x in xs]
    kk = [0.15, 0.15, 0.2, 0.2]
    I, tau, Iseq = 0.0, 0.0, []
    for k in range(4):
        I = I * math.exp(-kk[k] * ds) + jk[k] * math.exp(-tau) * ds
        tau += kk[k] * ds
        Iseq.append(I)
    # hand values of the first two substeps
    assert abs(Iseq[0] - 2.21875 * 0.5) < 1e-15
    assert abs(Iseq[1] - (1.109375 * math.exp(-0.075) + 2.46875 * math.exp(-0.075) * 0.5)) < 1e-15
    for geom in (0, 1):
        base, nn, Io = oracle.trace_ray(j[None], kap[None], src, 1, 0, ds, 4, geom_mode=geom)
        np.testing.assert_allclose(Io, Iseq, rtol=1e-14)
        cells = [np.ravel_multi_index((int(math.floor(x)), 1, 1), shape) for x in xs]
        assert list(base) == cells and list(nn) == cells
        F = oracle.advance(j[None], kap[None], src[None], 1, ds, 4, geom_mode=geom)[0]
        # tent-function form of the trilinear deposit: w_v(x) = prod_a max(0, 1 - |v_a - x_a|)
        expect = np.zeros(shape)
        for x0, Ik in zip(xs, Iseq):
            x = np.array([x0, 1.5, 1.75])
            expect += FOUR_PI * Ik * np.prod(np.maximum(0.0, 1.0 - np.abs(v - x)), axis=-1)
        np.testing.assert_allclose(F, expect, rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------------------------------------
# Linearity, sources, bins, shards (Sec. 2)
# --------------------------------------------------------------------------------------------
def test_linearity_in_j():
    p = inputs.random_small(3)
    rng = np.random.default_rng(0)
    j1 = p.j.astype(np.float64)
    j2 = rng.uniform(0, 1, p.j.shape)
    a, b = 0.37, -1.9
    F1 = oracle.advance(j1, p.kappa, p.sources, p.num_rays, p.step_size, 11)
    F2 = oracle.advance(j2, p.kappa, p.sources, p.num_rays, p.step_size, 11)
    F12 = oracle.advance(a * j1 + b * j2, p.kappa, p.sources, p.num_rays, p.step_size, 11)
    np.testing.assert_allclose(F12, a * F1 + b * F2, rtol=1e-12, atol=1e-12 * np.abs(F12).max())


def test_sources_loop_and_sum():
    p = inputs.random_small(4)
    F = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, 10)
    Fs = sum(oracle.advance(p.j, p.kappa, s[None], p.num_rays, p.step_size, 10) for s in p.sources)
    np.testing.assert_allclose(F, Fs, rtol=1e-13, atol=1e-14 * np.abs(F).max())


def test_bins_are_independent_batch():
    p = inputs.random_small(5, n_freq=3)
    F = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, 10)
    for b in range(3):
        Fb = oracle.advance(p.j[b:b + 1], p.kappa[b:b + 1], p.sources, p.num_rays, p.step_size, 10)
        assert np.array_equal(F[b], Fb[0])


def test_direction_shards_sum_to_whole():
    p = inputs.random_small(6)
    F = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, 10)
    cut = [0, 5, 20, p.num_rays]
    Fs = sum(oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, 10, ray_range=(a, b))
             for a, b in zip(cut[:-1], cut[1:]))
    np.testing.assert_allclose(F, Fs, rtol=1e-13, atol=1e-14 * np.abs(F).max())


# --------------------------------------------------------------------------------------------
# Horizon: finite light-travel distance (Sec. 1 goal (i); Sec. 2 N_s)
# --------------------------------------------------------------------------------------------
def test_light_travel_horizon():
    n, ds, horizon = 24, 0.5, 7.0
    ns = oracle.num_substeps(ds, 1.0, horizon)
    src = np.array([[11.3, 12.1, 10.7]])
    j = np.full((1, n, n, n), 0.5)
    kap = np.full((1, n, n, n), 0.05)
    F = oracle.advance(j, kap, src, 400, ds, ns)[0]
    r = np.linalg.norm(_grid_coords((n, n, n)) - src[0], axis=-1)
    reach = (ns - 1) * ds
    assert np.all(F[r > reach + math.sqrt(3) + 1e-9] == 0.0)
    # the front does get there: every direction deposits up to distance (N_s - 1) ds
    shell = (r > reach - 0.5) & (r <= reach + math.sqrt(3))
    assert np.count_nonzero(F[shell]) > 0.5 * np.count_nonzero(shell)


# --------------------------------------------------------------------------------------------
# Analytic point source, uniform kappa (Sec. 3 "Analytical validation", Eq. 3)
# --------------------------------------------------------------------------------------------
def _analytic_case(nr, ds, n=32, horizon=16.0, kap=0.1):
    p = inputs.single_source_uniform(n=n, kappa0=kap, sigma=1.0, num_rays=nr, step_size=ds,
                                     horizon=horizon)
    ns = oracle.num_substeps(ds, 1.0, horizon)
    F = oracle.advance(p.j, p.kappa, p.sources, nr, ds, ns, geom_mode=1)[0]
    c = p.sources[0].astype(np.float64)
    r = np.linalg.norm(_grid_coords((n, n, n)) - c, axis=-1)
    # Luminosity normalisation: on each ray the recursion gives
    # I_{k+1} = exp(-kappa k ds) ds sum_{m<=k} j(x_m); deposits are N_Omega / (4 pi r^2 ds) per
    # unit volume, so J(r) = S exp(-kappa r) / r^2 with S the ray average of sum_m j(x_m),
    # i.e. L / (4 pi) = S. S is evaluated with scipy's trilinear interpolation (order 1,
    # nearest-edge), independently of the oracle.
    d = oracle.fibonacci_dirs(nr)
    pts = c[None, None, :] + np.arange(ns)[None, :, None] * ds * d[:, None, :]
    jm = map_coordinates(p.j[0].astype(np.float64), pts.reshape(-1, 3).T, order=1, mode="nearest")
    S = jm.reshape(nr, ns).sum(1).mean()
    Jref = S * np.exp(-kap * r) / np.maximum(r, 1e-12) ** 2
    inner = np.zeros((n, n, n), bool)
    inner[1:-1, 1:-1, 1:-1] = True                         # drop a one-voxel border
    mask = inner & (r >= 2.0) & (r <= horizon - 2.0)       # drop the centre, stay in the horizon
    return F, Jref, r, mask


def test_analytic_point_source_shape():
    """Shell averages of F / J_ref - 1 stay within 2 % from r = 4 to the horizon: pins the
    1/r^2 geometry, the exp(-kappa r) attenuation and the exp(-tau_k) emission factor."""
    F, Jref, r, mask = _analytic_case(3072, 0.5)
    for lo in range(4, 14, 2):
        m = mask & (r >= lo) & (r < lo + 2)
        bias = np.mean(F[m] / Jref[m] - 1.0)
        assert abs(bias) < 0.02, (lo, bias)
    err = np.mean(np.abs(F[mask] - Jref[mask]) / Jref[mask])
    # the paper's average relative error against Eq. 3 (its N_Omega and ds are not stated): the
    # oracle with N_Omega 3072, ds 0.5 and the same exclusions is at least as close
    assert err <= PAPER["analytic_validation"]["mean_relative_error"], err


def test_timing_run_recipe_matches_the_printed_workload():
    """The synthetic stand-in for the paper's timing run has its printed shape: a 128^3 grid, 4,096
    rays and 2,097 sources, the 0.1 % highest-kappa cells (Sec. 2 timing, Sec. 3 source placement)."""
    t = PAPER["timing_run"]
    p = inputs.paper_timing()
    assert p.shape == (t["grid_edge"],) * 3
    assert p.num_rays == t["num_rays"]
    assert len(p.sources) == t["num_sources"]
    assert len(p.sources) == round(PAPER["turbulent_sources"]["fraction_of_cells"] * t["grid_edge"] ** 3)
    # the sources are the highest-kappa cells: every source cell's kappa >= every other cell's
    kap = p.kappa[0]
    idx = tuple(p.sources.astype(int).T)
    others = np.ones(kap.shape, bool)
    others[idx] = False
    assert kap[idx].min() >= kap[others].max()


def test_analytic_convergence_monotone():
    """Error vs Eq. 3 decreases monotonically in N_Omega and in ds (Sec. 3). In ds the error
    reaches its floor (angular sampling and the trilinear kernel) near ds = 0.5, so the ds
    sequence is 2, 1, 0.5."""
    def err(nr, ds):
        F, Jref, r, mask = _analytic_case(nr, ds)
        return np.mean(np.abs(F[mask] - Jref[mask]) / Jref[mask])
    e_rays = [err(nr, 0.5) for nr in (192, 768, 3072, 12288)]
    assert all(a > b for a, b in zip(e_rays[:-1], e_rays[1:])), e_rays
    e_ds = [err(3072, ds) for ds in (2.0, 1.0, 0.5)]
    assert all(a > b for a, b in zip(e_ds[:-1], e_ds[1:])), e_ds


# --------------------------------------------------------------------------------------------
# Axis order and the kappa convention
# --------------------------------------------------------------------------------------------
def test_absorbing_slab_shadows_along_axis0():
    """A slab of kappa = 5 at axis-0 index >= 13 shadows the +axis-0 side of a centred source
    only: pins the flat index order [axis0][axis1][axis2]."""
    n = 21
    v = _grid_coords((n, n, n))
    src = np.array([10.0, 10.0, 10.0])
    j = np.exp(-np.sum((v - src) ** 2, -1) / 2.0)[None]
    kap = np.where(v[..., 0] >= 13, 5.0, 0.01)[None]
    F = oracle.advance(j, kap, src[None], 768, 0.5, 18)[0]
    assert F[16, 10, 10] < 1e-3 * F[4, 10, 10]
    np.testing.assert_allclose(F[10, 16, 10], F[10, 4, 10], rtol=0.05)
    np.testing.assert_allclose(F[10, 10, 16], F[10, 10, 4], rtol=0.05)


def test_kappa_nearest_neighbour_convention():
    """kappa_mode 0 samples the clamped floor cell of the previous position x_k; kappa_mode 1
    the clamped round-to-nearest cell (reading R3: the paper does not fix which)."""
    shape = (10, 5, 5)
    v = _grid_coords(shape)
    kap = np.where(v[..., 0] >= 5, 10.0, 0.0)[None]
    j = np.ones((1,) + shape)
    src = np.array([3.25, 2.0, 2.0])
    # x0 = 3.25, 3.75, 4.25, 4.75, 5.25: floor 3,3,4,4,5 ; round 3,4,4,5,5
    _, nn0, I0 = oracle.trace_ray(j, kap, src, 1, 0, 0.5, 6, kappa_mode=0)
    _, nn1, I1 = oracle.trace_ray(j, kap, src, 1, 0, 0.5, 6, kappa_mode=1)
    assert [np.unravel_index(c, shape)[0] for c in nn0] == [3, 3, 4, 4, 5, 5]
    assert [np.unravel_index(c, shape)[0] for c in nn1] == [3, 4, 4, 5, 5, 6]
    np.testing.assert_allclose(I0[:4], 0.5 * np.arange(1, 5), rtol=1e-15)   # kappa 0 until k=4
    np.testing.assert_allclose(I1[:3], 0.5 * np.arange(1, 4), rtol=1e-15)   # kappa 0 until k=3
    assert I0[4] < I0[3] and I1[3] < I1[2]


# --------------------------------------------------------------------------------------------
# Brute force on a 4^3 grid: double-sum form of the recursion, scipy interpolation
# --------------------------------------------------------------------------------------------
def _brute_force_response(kappa, src, nr, ds, ns):
    """Linear response M (F = M j, fixed kappa) of the whole operator on a tiny grid, from the
    non-recursive form I_{k+1} = sum_{m<=k} j_m ds exp(-tau_m) exp(-(tau_{k+1} - tau_{m+1}))
    with j_m and the deposit weights taken from scipy's map_coordinates (order 1, clamped),
    and geometry in FP32 as reading R6 prescribes."""
    shape = kappa.shape
    nc = kappa.size
    dirs = oracle.fibonacci_dirs(nr).astype(np.float32)
    ds = float(np.float32(ds))      # parity mode: the step length is an FP32 value
    imp = np.eye(nc).reshape((nc,) + shape)
    M = np.zeros((nc, nc))
    for s in src:
        for d in dirs:
            dd = (d * np.float32(ds)).astype(np.float32)
            x = np.asarray(s, np.float32)
            xs = []
            for _ in range(ns):
                xs.append(x.astype(np.float64))
                x = (x + dd).astype(np.float32)
            xs = np.array(xs)
            cell = np.clip(np.floor(xs).astype(int), 0, np.array(shape) - 1)
            kk = kappa[cell[:, 0], cell[:, 1], cell[:, 2]]
            tau = np.concatenate([[0.0], np.cumsum(kk * ds)])
            W = np.stack([map_coordinates(imp[u], xs.T, order=1, mode="nearest") for u in range(nc)])
            # coefficient of j_m in I_{k+1}
            C = np.zeros((ns, ns))
            for k in range(ns):
                for m in range(k + 1):
                    C[k, m] = ds * math.exp(-tau[m]) * math.exp(-(tau[k + 1] - tau[m + 1]))
            M += (FOUR_PI / nr) * W @ C @ W.T
    return M


def test_brute_force_4cubed_response_matrix():
    rng = np.random.default_rng(7)
    shape = (4, 4, 4)
    kappa = rng.uniform(0.0, 0.8, shape)
    src = np.array([[1.3, 2.2, 1.7], [3.6, 0.4, 2.9]])
    nr, ds, ns = 6, 0.7, 7
    M = _brute_force_response(kappa, src, nr, ds, ns)
    Mo = np.zeros_like(M)
    for u in range(64):
        e = np.zeros(64)
        e[u] = 1.0
        Mo[:, u] = oracle.advance(e.reshape((1,) + shape), kappa[None], src, nr, ds, ns)[0].ravel()
    np.testing.assert_allclose(Mo, M, rtol=1e-11, atol=1e-13 * np.abs(M).max())


# --------------------------------------------------------------------------------------------
# Adjoint (reverse mode of Eq. 2) -- Sec. 4 says the Jacobians w.r.t. (j, kappa) are defined
# --------------------------------------------------------------------------------------------
def test_adjoint_j_dot_product():
    """F is linear in j, so <G, F(dj)> = <F^T G, dj> must hold to rounding."""
    p = inputs.random_small(8, n_freq=2)
    rng = np.random.default_rng(1)
    G = rng.standard_normal(p.j.shape)
    dj = rng.standard_normal(p.j.shape)
    Fd = oracle.advance(dj, p.kappa, p.sources, p.num_rays, p.step_size, 12)
    gj, _ = oracle.backward(p.j, p.kappa, p.sources, p.num_rays, p.step_size, 12, G)
    lhs, rhs = np.sum(G * Fd), np.sum(gj * dj)
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(G * Fd).sum())


def test_adjoint_matches_brute_force_transpose():
    rng = np.random.default_rng(9)
    shape = (4, 4, 4)
    kappa = rng.uniform(0.0, 0.8, shape)
    src = np.array([[1.3, 2.2, 1.7]])
    M = _brute_force_response(kappa, src, 5, 0.7, 6)
    G = rng.standard_normal(64)
    gj, _ = oracle.backward(np.zeros((1,) + shape), kappa[None], src, 5, 0.7, 6, G.reshape((1,) + shape))
    np.testing.assert_allclose(gj.ravel(), M.T @ G, rtol=1e-11, atol=1e-13 * np.abs(M.T @ G).max())


@pytest.mark.parametrize("geom", [0, 1])
def test_adjoint_kappa_central_fd(geom):
    """FP64 central differences, h = 1e-6, on a 16^3 lognormal medium with N_Omega = 192."""
    n = 16
    kap = inputs.lognormal_field((n, n, n), 1.0, 0.05, 41).astype(np.float64)[None]
    v = _grid_coords((n, n, n))
    src = np.array([[7.3, 8.1, 6.6], [3.0, 11.5, 9.2]])
    j = sum(np.exp(-np.sum((v - s) ** 2, -1) / 8.0) for s in src)[None]
    nr, ds, ns = 192, 0.5, 20
    rng = np.random.default_rng(3)
    G = rng.standard_normal(j.shape)
    _, gk = oracle.backward(j, kap, src, nr, ds, ns, G, geom_mode=geom)
    h = 1e-6
    for trial in range(3):
        e = rng.standard_normal(kap.shape)
        Lp = np.sum(G * oracle.advance(j, kap + h * e, src, nr, ds, ns, geom_mode=geom))
        Lm = np.sum(G * oracle.advance(j, kap - h * e, src, nr, ds, ns, geom_mode=geom))
        fd = (Lp - Lm) / (2 * h)
        ad = np.sum(gk * e)
        assert abs(fd - ad) <= 1e-6 * abs(ad) + 1e-9, (trial, fd, ad)
    # single voxels that a ray crosses
    for idx in [(0, 7, 8, 6), (0, 9, 8, 7), (0, 3, 10, 9)]:
        e = np.zeros_like(kap)
        e[idx] = 1.0
        Lp = np.sum(G * oracle.advance(j, kap + h * e, src, nr, ds, ns, geom_mode=geom))
        Lm = np.sum(G * oracle.advance(j, kap - h * e, src, nr, ds, ns, geom_mode=geom))
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - gk[idx]) <= 1e-6 * abs(gk[idx]) + 1e-9


# --------------------------------------------------------------------------------------------
# Inversion (Sec. 4, "Gradient-based inversion"): scalar amplitude with a fixed template
# --------------------------------------------------------------------------------------------
def test_amplitude_inversion_reaches_closed_form():
    """F(A e0) = A F(e0), so the MSE minimiser is A* = <F0, I_ref> / <F0, F0> and the
    relative-MSE one A* = sum(F0 I / I^2) / sum(F0^2 / I^2). Gradient descent on A with
    dL/dA = <dL/dj, e0> from the adjoint must land on both."""
    n = 12
    v = _grid_coords((n, n, n))
    src = np.array([[5.5, 5.5, 5.5]])
    e0 = np.exp(-np.sum((v - src[0]) ** 2, -1) / 2.0)[None]
    kap = np.full_like(e0, 0.1)
    nr, ds, ns = 96, 0.5, 14
    F0 = oracle.advance(e0, kap, src, nr, ds, ns)
    rng = np.random.default_rng(5)
    Iref = 2.7 * F0 * (1.0 + 0.05 * rng.standard_normal(F0.shape))
    pos = Iref > 0
    for kind in ("mse", "rel"):
        wgt = np.where(pos, 1.0, 0.0) if kind == "mse" else np.where(pos, 1.0 / np.where(pos, Iref, 1.0) ** 2, 0.0)
        A_star = np.sum(wgt * F0 * Iref) / np.sum(wgt * F0 * F0)
        A = 0.0
        curv = 2.0 * np.sum(wgt * F0 * F0)
        for _ in range(30):
            G = 2.0 * wgt * (oracle.advance(A * e0, kap, src, nr, ds, ns) - Iref)
            gj, _ = oracle.backward(A * e0, kap, src, nr, ds, ns, G)
            A -= 0.8 * np.sum(gj * e0) / curv
        assert abs(A - A_star) <= 1e-8 * abs(A_star), (kind, A, A_star)
