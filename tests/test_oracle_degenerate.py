"""Pins of the FP64 oracle on degenerate grids (no GPU): extents of one or two cells.

A single-cell axis clamps both trilinear corners to its one cell (Sec. 2: indices clamped to
the box), so such a grid must equal the same medium laid out as two identical layers along
that axis with the deposits of the two layers summed; a 1 x 1 x 1 grid holds every deposit of
every ray and must equal the closed form of Eq. 2 for a uniform medium.
"""
import math

import numpy as np
import pytest

import oracle

FOUR_PI = 4.0 * math.pi


def _arith_geo(a, n):
    """sum_{m=1}^{n} m a^(m-1), by its closed form (1 - (n+1) a^n + n a^(n+1)) / (1 - a)^2."""
    if a == 1.0:
        return n * (n + 1) / 2.0
    return (1.0 - (n + 1) * a ** n + n * a ** (n + 1)) / (1.0 - a) ** 2


def test_single_cell_grid_closed_form():
    """Uniform j, kappa in one cell: E_k = a^k with a = exp(-kappa ds), so I_{k+1} = (k+1) j ds a^k
    for every ray, and the cell receives 4 pi N_src j ds sum_{m=1}^{N_s} m a^(m-1)."""
    j0 = np.array([0.7, 0.2, 1.3])
    k0 = np.array([0.3, 0.05, 0.0])
    j = j0[:, None, None, None] * np.ones((3, 1, 1, 1))
    kappa = k0[:, None, None, None] * np.ones((3, 1, 1, 1))
    src = np.array([[0.2, -0.4, 0.9], [3.5, 0.0, -2.0], [0.0, 0.0, 0.0]])   # in, outside, on the cell
    ds, ns, nr = 0.5, 40, 24
    for geom in (0, 1):
        F = oracle.advance(j, kappa, src, nr, ds, ns, geom_mode=geom)
        for b in range(3):
            expect = FOUR_PI * len(src) * j0[b] * ds * _arith_geo(math.exp(-k0[b] * ds), ns)
            assert F[b, 0, 0, 0] == pytest.approx(expect, rel=1e-12), (geom, b)


@pytest.mark.parametrize("axes", [(0,), (1,), (2,), (1, 2), (0, 2)])
def test_single_cell_axes_equal_summed_identical_layers(axes):
    """Extent 1 along `axes` vs extent 2 with two identical layers, summed over those axes: the
    trilinear weights along a duplicated axis sum to one, and a clamped axis puts both on one cell."""
    rng = np.random.default_rng(17 + sum(axes))
    base = [9, 7, 8]
    thin = [1 if a in axes else n for a, n in enumerate(base)]
    j1 = rng.uniform(0.0, 1.0, (2,) + tuple(thin))
    k1 = rng.uniform(0.0, 0.5, (2,) + tuple(thin))
    reps = [1] + [2 if a in axes else 1 for a in range(3)]
    j2, k2 = np.tile(j1, reps), np.tile(k1, reps)
    src = np.stack([rng.uniform(-1.5, n + 0.5, 4) for n in thin], axis=1)
    for kappa_mode in (0, 1):
        A = oracle.advance(j1, k1, src, 30, 0.6, 21, kappa_mode=kappa_mode)
        B = oracle.advance(j2, k2, src, 30, 0.6, 21, kappa_mode=kappa_mode)
        Bs = B.sum(axis=tuple(a + 1 for a in axes), keepdims=True)
        np.testing.assert_allclose(A, Bs, rtol=1e-11, atol=1e-13 * np.abs(A).max())


def test_two_cell_axes_weights_and_adjoint_dot_product():
    """Extent 2 along every axis (every corner set is the whole grid): the field is linear in j,
    so the adjoint satisfies <G, F(dj)> = <F^T G, dj>, and the total deposit equals the
    uniform-medium closed form when j and kappa are uniform."""
    rng = np.random.default_rng(5)
    shape = (1, 2, 2, 2)
    kappa = rng.uniform(0.0, 0.6, shape)
    src = np.array([[0.4, 0.7, 0.2], [-1.0, 1.5, 0.5]])
    G = rng.standard_normal(shape)
    dj = rng.standard_normal(shape)
    Fd = oracle.advance(dj, kappa, src, 18, 0.5, 15)
    gj, _ = oracle.backward(np.zeros(shape), kappa, src, 18, 0.5, 15, G)
    assert abs(np.sum(G * Fd) - np.sum(gj * dj)) <= 1e-12 * np.abs(G * Fd).sum()
    F = oracle.advance(np.full(shape, 0.9), np.full(shape, 0.25), src, 18, 0.5, 15)
    expect = FOUR_PI * len(src) * 0.9 * 0.5 * _arith_geo(math.exp(-0.25 * 0.5), 15)
    assert F.sum() == pytest.approx(expect, rel=1e-12)


def test_single_cell_axis_adjoint_central_fd():
    """dL/dkappa of the oracle's reverse march on a slab one cell thick against FP64 central
    differences of its forward march."""
    rng = np.random.default_rng(23)
    shape = (1, 6, 1, 5)
    j = rng.uniform(0.1, 1.0, shape)
    kap = rng.uniform(0.05, 0.6, shape)
    src = np.array([[2.3, 0.1, 1.8], [4.0, -0.7, 3.1]])
    nr, ds, ns = 40, 0.5, 14
    G = rng.standard_normal(shape)
    gj, gk = oracle.backward(j, kap, src, nr, ds, ns, G)
    h = 1e-6
    for trial in range(3):
        e = rng.standard_normal(shape)
        Lp = np.sum(G * oracle.advance(j, kap + h * e, src, nr, ds, ns))
        Lm = np.sum(G * oracle.advance(j, kap - h * e, src, nr, ds, ns))
        fd = (Lp - Lm) / (2 * h)
        ad = np.sum(gk * e)
        assert abs(fd - ad) <= 1e-6 * abs(ad) + 1e-9, (trial, fd, ad)
    # and dL/dj is exact: F is linear in j
    e = rng.standard_normal(shape)
    lin = np.sum(G * oracle.advance(e, kap, src, nr, ds, ns))
    assert abs(lin - np.sum(gj * e)) <= 1e-12 * np.abs(lin) + 1e-14


def test_source_gradient_on_a_slab():
    """dL/d(source position) on a slab one cell thick along axis 1: the component along that axis
    vanishes (both corners are the one cell, for the gather and the deposit alike: its terms
    cancel to rounding), and the other two match FP64 central differences of the march."""
    from paper_2511_09389_gb300 import inputs
    rng = np.random.default_rng(31)
    p = inputs.random_small(31, shape=(10, 1, 9), n_freq=2, n_src=2, num_rays=48, step_size=0.6, horizon=5.0,
                            outside=False)
    ns = oracle.num_substeps(p.step_size, 1.0, p.time_step)
    G = rng.standard_normal(p.j.shape)
    src = p.sources.astype(np.float64)
    src[:, 1] = [0.3, -0.8]                      # inside the one cell and outside it

    def loss(s):
        return float((G * oracle.advance(p.j, p.kappa, s, p.num_rays, p.step_size, ns, geom_mode=1)).sum())

    g = oracle.source_gradient(p.j, p.kappa, src, p.num_rays, p.step_size, ns, G, geom_mode=1)
    assert np.abs(g[:, 1]).max() <= 1e-12 * np.abs(g).max()
    h = 1e-6
    fd = np.zeros_like(src)
    for s in range(src.shape[0]):
        for a in (0, 2):
            e = np.zeros_like(src)
            e[s, a] = h
            fd[s, a] = (loss(src + e) - loss(src - e)) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-7 * np.abs(fd).max()
