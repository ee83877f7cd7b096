"""Pins of the oracle's stateful advance (the march continued across calls: time integration with a fixed dt,
Sec. 3): a restart is the plain advance, consecutive calls add up to one longer call, and a
call through an empty, transparent medium deposits exactly the carried intensity."""
import numpy as np
import pytest

import oracle
from paper_2511_09389_gb300 import inputs


@pytest.fixture(scope="module")
def prob():
    return inputs.random_small(8, shape=(12, 10, 14), n_freq=2, n_src=3, num_rays=96, step_size=0.5, horizon=8.0)


def test_restart_is_the_plain_advance(prob):
    p = prob
    st = oracle.MarchState(p.n_freq, len(p.sources), p.num_rays)
    st.pos[:] = 123.0      # ignored on restart
    F = oracle.advance_state(p.j, p.kappa, p.sources, p.num_rays, p.step_size, 16, st, restart=True)
    R = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, 16)
    assert np.array_equal(F, R)


@pytest.mark.parametrize("split", [(16, 16), (5, 27), (1, 9, 22)])
def test_consecutive_calls_add_up_to_one_call(prob, split):
    p = prob
    total = sum(split)
    st = oracle.MarchState(p.n_freq, len(p.sources), p.num_rays)
    parts = [oracle.advance_state(p.j, p.kappa, p.sources, p.num_rays, p.step_size, n, st, restart=(i == 0))
             for i, n in enumerate(split)]
    one = oracle.MarchState(p.n_freq, len(p.sources), p.num_rays)
    R = oracle.advance_state(p.j, p.kappa, p.sources, p.num_rays, p.step_size, total, one, restart=True)
    assert np.abs(sum(parts) - R).max() <= 1e-12 * np.abs(R).max()
    # the carried state is the one-call state, operation for operation
    assert np.array_equal(st.pos, one.pos) and np.array_equal(st.I, one.I) and np.array_equal(st.tau, one.tau)
    assert np.array_equal(R, oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, total))


def test_transparent_empty_call_deposits_the_carried_intensity(prob):
    """j = 0, kappa = 0: I stays at its carried value, so each bin's field sums (weights sum to
    one, also clamped) to 4 pi / N_Omega * n_steps * sum over rays of I."""
    p = prob
    st = oracle.MarchState(p.n_freq, len(p.sources), p.num_rays)
    oracle.advance_state(p.j, p.kappa, p.sources, p.num_rays, p.step_size, 10, st, restart=True)
    I_end = st.I.copy()
    pos = st.pos.copy()
    z = np.zeros_like(p.j)
    F = oracle.advance_state(z, z, p.sources, p.num_rays, p.step_size, 7, st, restart=False)
    expect = 4.0 * np.pi / p.num_rays * 7 * I_end.reshape(p.n_freq, -1).sum(axis=1)
    assert np.allclose(F.reshape(p.n_freq, -1).sum(axis=1), expect, rtol=1e-12)
    assert np.array_equal(st.I, I_end) and np.all(st.tau == st.tau)
    # positions moved by 7 FP32 steps along each ray
    d = (oracle.fibonacci_dirs_f32(p.num_rays) * np.float32(p.step_size)).astype(np.float32)
    x = pos.astype(np.float32)
    for _ in range(7):
        x = (x + d[None]).astype(np.float32)
    assert np.array_equal(st.pos, x.astype(np.float64))
