"""The oracle's threaded driver computes the same field as the one-thread oracle.

The field is a sum over (source, ray) items, so only the order of FP64 additions changes:
agreement to 1e-13 relative, bit-equal across runs with the same thread count and block, and
shards of the lattice still add up to the whole.
"""
import numpy as np
import pytest

import oracle
from paper_2511_09389_gb300 import inputs


@pytest.fixture(scope="module")
def prob():
    p = inputs.random_small(3, shape=(20, 18, 16), n_freq=3, n_src=5, num_rays=300, horizon=16.0)
    ns = oracle.num_substeps(p.step_size, 1.0, p.time_step)
    return p, ns, oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns)


@pytest.mark.parametrize("threads,block", [(2, 64), (3, 37), (8, 300), (16, 1)])
def test_threads_match_one_thread(prob, threads, block):
    p, ns, ref = prob
    a = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns, threads=threads, ray_block=block)
    b = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns, threads=threads, ray_block=block)
    assert np.abs(a - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.array_equal(a, b)


def test_threaded_shards_sum_to_whole(prob):
    p, ns, ref = prob
    parts = [oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns, ray_range=r, threads=4,
                            ray_block=50) for r in [(0, 111), (111, 300)]]
    assert np.abs(parts[0] + parts[1] - ref).max() <= 1e-13 * np.abs(ref).max()


def test_threaded_rejects_bad_arguments(prob):
    p, ns, _ = prob
    with pytest.raises(ValueError):
        oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns, threads=4, ray_block=0)
    with pytest.raises(ValueError):
        oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns, ray_range=(0, 301), threads=4)
