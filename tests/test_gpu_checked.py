"""Checked mode (rt_options.check_inputs), the one-shot batch (rt_advance_batch) and
rt_sync_status."""
import ctypes

import numpy as np
import pytest

from paper_2511_09389_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2511_09389_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


def test_checked_mode_names_the_bad_input(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Grid, RTError
    p = inputs.random_small(31, shape=(10, 9, 12), n_freq=3, n_src=2, num_rays=64, horizon=6.0)
    j, k, s = (torch.from_numpy(a).cuda() for a in (p.j, p.kappa, p.sources))
    gc = Grid(p.shape, 8, check_inputs=True)
    g = Grid(p.shape, 8)
    a = gc.advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step).cpu().numpy()
    b = g.advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step).cpu().numpy()
    assert np.allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max())
    cases = []
    jj = j.clone(); jj[1, 3, 4, 5] = float("nan"); cases.append((jj, k, s, "j_map"))
    kk = k.clone(); kk[2, 0, 0, 0] = -0.25; cases.append((j, kk, s, "kappa_map"))
    kk2 = k.clone(); kk2[0, 9, 8, 11] = float("inf"); cases.append((j, kk2, s, "kappa_map"))
    ss = s.clone(); ss[1, 2] = float("nan"); cases.append((j, k, ss, "source_pos"))
    ss2 = s.clone(); ss2[0, 0] = 3.0e7; cases.append((j, k, ss2, "source_pos"))
    for jx, kx, sx, name in cases:
        with pytest.raises(RTError, match=name):
            gc.advance(jx, kx, sx, p.num_rays, p.step_size, 1.0, p.time_step)
        g.advance(jx, kx, sx, p.num_rays, p.step_size, 1.0, p.time_step)      # unchecked: no scan
    G = torch.randn_like(j)
    G[0, 1, 1, 1] = float("nan")
    with pytest.raises(RTError, match="grad_out"):
        gc.backward(G, j, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
    from paper_2511_09389_gb300 import _native
    torch.cuda.synchronize()
    assert _native.load().rt_sync_status(None) == 0


def test_one_shot_batch_matches_single_calls(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300 import _native
    from paper_2511_09389_gb300.api import Grid
    lib = _native.load()
    probs = inputs.batch_instances(6, seed=3200, edges=(16, 24, 32), ray_choices=(192, 768), max_src=4, max_freq=5)
    arr = (_native.rt_instance * len(probs))()
    keep, outs = [], []
    for i, p in enumerate(probs):
        j, k, s = (torch.from_numpy(a).cuda() for a in (p.j, p.kappa, p.sources))
        out = torch.full_like(j, 7.0)
        keep += [j, k, s, out]
        outs.append(out)
        nf, n0, n1, n2 = j.shape
        arr[i] = _native.rt_instance(j.data_ptr(), k.data_ptr(), s.data_ptr(), s.shape[0], n0, n1, n2, nf,
                                     p.num_rays, p.step_size, 1.0, p.time_step, out.data_ptr())
    g = Grid((8, 8, 8), 8)
    assert lib.rt_advance_batch(g._h, arr, len(probs), None) == 0, lib.rt_last_error()
    for p, out, (j, k, s) in zip(probs, outs, [keep[4 * i:4 * i + 3] for i in range(len(probs))]):
        ref = Grid(p.shape, 8).advance(j, k, s, p.num_rays, p.step_size, 1.0, p.time_step)
        assert float((out - ref).norm() / ref.norm()) <= 1e-5
    assert lib.rt_sync_status(None) == 0
