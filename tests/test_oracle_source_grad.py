"""Pins of the oracle's gradient with respect to the source positions: central finite
differences of the FP64 march, a uniform medium (the loss does not depend on where the
sources are) and a closed form for an affine emission field in a transparent medium."""
import numpy as np
import pytest

import oracle
from paper_2511_09389_gb300 import inputs


def loss(p, src, G, ns):
    return float((G * oracle.advance(p.j, p.kappa, src, p.num_rays, p.step_size, ns, geom_mode=1)).sum())


@pytest.mark.parametrize("seed", [5, 6])
def test_matches_central_differences(seed):
    rng = np.random.default_rng(seed)
    p = inputs.random_small(seed, shape=(10, 9, 11), n_freq=2, n_src=2, num_rays=48, step_size=0.6, horizon=5.0,
                            outside=False)
    ns = oracle.num_substeps(p.step_size, 1.0, p.time_step)
    G = rng.standard_normal(p.j.shape)
    src = p.sources.astype(np.float64)
    g = oracle.source_gradient(p.j, p.kappa, src, p.num_rays, p.step_size, ns, G, geom_mode=1)
    h = 1e-6
    fd = np.zeros_like(src)
    for s in range(src.shape[0]):
        for a in range(3):
            e = np.zeros_like(src)
            e[s, a] = h
            fd[s, a] = (loss(p, src + e, G, ns) - loss(p, src - e, G, ns)) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-7 * np.abs(fd).max()


def test_uniform_medium_gives_zero():
    shape = (12, 12, 12)
    j = np.full((1,) + shape, 0.7)
    k = np.full((1,) + shape, 0.05)
    src = np.array([[5.3, 6.1, 4.7], [2.2, 9.5, 7.75]])
    G = np.ones((1,) + shape)
    g = oracle.source_gradient(j, k, src, 64, 0.5, 12, G, geom_mode=1)
    assert np.abs(g).max() <= 1e-10


def test_affine_emission_closed_form():
    """j = alpha x_0 + beta, kappa = 0, G = 1, rays inside the box: L = s ds sum_rays
    sum_m (N_s - m) j(x_m), so dL/dsrc_0 = 4 pi ds alpha N_s (N_s + 1) / 2 and the other two
    components vanish."""
    n, alpha, beta, ds, ns = 24, 0.3, 2.0, 0.5, 14
    x0 = np.arange(n, dtype=np.float64)[:, None, None]
    j = (alpha * x0 + beta) * np.ones((1, n, n, n))
    k = np.zeros_like(j)
    src = np.array([[11.3, 11.6, 11.45]])
    G = np.ones_like(j)
    g = oracle.source_gradient(j, k, src, 96, ds, ns, G, geom_mode=1)
    expect = 4.0 * np.pi * ds * alpha * ns * (ns + 1) / 2
    assert g[0, 0] == pytest.approx(expect, rel=1e-12)
    assert abs(g[0, 1]) <= 1e-9 * expect and abs(g[0, 2]) <= 1e-9 * expect
