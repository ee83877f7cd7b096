"""Batched persistent launch (rt_batch_*): every instance of a batch equals its own
rt_advance (and the oracle), across graph replays and in-place input updates."""
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


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def small_instances():
    out = []
    for i, (shape, nf, nsrc, rays, ds, hz) in enumerate([((12, 10, 14), 1, 3, 64, 0.5, 9.0),
                                                         ((16, 16, 16), 4, 2, 200, 0.5, 14.0),
                                                         ((9, 13, 7), 2, 5, 33, 0.75, 8.0),
                                                         ((20, 8, 11), 5, 1, 96, 0.6, 12.0),
                                                         ((8, 8, 8), 3, 4, 300, 0.5, 6.0),
                                                         ((24, 20, 18), 8, 2, 130, 0.5, 16.0)]):
        out.append(inputs.random_small(200 + i, shape=shape, n_freq=nf, n_src=nsrc, num_rays=rays,
                                       step_size=ds, horizon=hz))
    return out


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_matches_per_instance_and_oracle(torch_cuda, autotune):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Batch, Grid
    probs = small_instances()
    dev = [{k: torch.from_numpy(v).cuda() for k, v in (("j", p.j), ("kappa", p.kappa), ("sources", p.sources))}
           for p in probs]
    for d, p in zip(dev, probs):
        d.update(num_rays=p.num_rays, step_size=p.step_size, radiation_velocity=1.0, time_step=p.time_step)
    b = Batch(dev, autotune=autotune)
    assert b.updates == sum(len(p.sources) * p.num_rays * oracle.num_substeps(p.step_size, 1.0, p.time_step)
                            * p.n_freq for p in probs)
    for rep in range(2):                                 # capture, then a graph replay
        outs = [o.cpu().numpy() for o in b.run()]
        torch.cuda.synchronize()
        for p, d, F in zip(probs, dev, outs):
            g = Grid(p.shape, 8)
            single = g.advance(d["j"], d["kappa"], d["sources"], p.num_rays, p.step_size, 1.0, p.time_step)
            assert rel(F, single.cpu().numpy()) <= 1e-5
            R = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size,
                               oracle.num_substeps(p.step_size, 1.0, p.time_step))
            for bb in range(p.n_freq):
                assert rel(F[bb], R[bb]) <= 1e-5
    # inputs updated in place are picked up by the next replay
    dev[1]["j"].mul_(2.0)
    F2 = b.run()[1].cpu().numpy()
    torch.cuda.synchronize()
    np.testing.assert_allclose(F2, 2 * outs[1], rtol=1e-5, atol=1e-6 * np.abs(outs[1]).max())
    b.close()


@pytest.mark.parametrize("autotune", [False, True])
def test_mixed_batch_dedicated_and_persistent(torch_cuda, autotune):
    """Instances with at least RT_BATCH_DEDICATED_LANES (source, ray, bin group) lanes get their own
    launches (a 4-bin group pair and a one-bin instance here, just above the threshold of 19,456);
    the rest share the persistent kernels. Every output equals its own rt_advance and the oracle."""
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Batch, Grid
    big4 = inputs.random_small(240, shape=(20, 18, 16), n_freq=5, n_src=3, num_rays=3300, step_size=0.5,
                               horizon=10.0)     # 3 x 3300 x 2 groups = 19,800 lanes
    big1 = inputs.random_small(241, shape=(17, 15, 19), n_freq=1, n_src=7, num_rays=2800, step_size=0.5,
                               horizon=8.0)      # 7 x 2800 = 19,600 lanes
    probs = [small_instances()[1], big4, small_instances()[0], big1, small_instances()[3]]
    dev = [{k: torch.from_numpy(v).cuda() for k, v in (("j", p.j), ("kappa", p.kappa), ("sources", p.sources))}
           for p in probs]
    for d, p in zip(dev, probs):
        d.update(num_rays=p.num_rays, step_size=p.step_size, radiation_velocity=1.0, time_step=p.time_step)
    b = Batch(dev, autotune=autotune)
    for rep in range(2):
        outs = [o.cpu().numpy() for o in b.run()]
        torch.cuda.synchronize()
        for p, d, F in zip(probs, dev, outs):
            g = Grid(p.shape, 8)
            single = g.advance(d["j"], d["kappa"], d["sources"], p.num_rays, p.step_size, 1.0, p.time_step)
            assert rel(F, single.cpu().numpy()) <= 1e-5
            R = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size,
                               oracle.num_substeps(p.step_size, 1.0, p.time_step))
            for bb in range(p.n_freq):
                assert rel(F[bb], R[bb]) <= 1e-5
    info = [b.info(i) for i in range(len(probs))]
    assert [x["dedicated"] for x in info] == [0, 1, 0, 1, 0]
    assert info[3]["bins_per_thread"] == 1
    assert info[1]["bins_per_thread"] in ((1, 2, 4) if autotune else (4,))
    assert all(x["block"] in (32, 64, 128, 256) for x in info)
    b.close()


def test_batch_rejects_bad_instances(torch_cuda):
    torch = torch_cuda
    from paper_2511_09389_gb300.api import Batch, RTError
    j = torch.ones(1, 4, 4, 4, device="cuda")
    base = dict(j=j, kappa=j.clone(), sources=torch.zeros(1, 3, device="cuda"), num_rays=8, step_size=0.5,
                time_step=2.0)
    for bad in (dict(num_rays=0), dict(step_size=0.0), dict(time_step=-1.0), dict(sources=torch.zeros(0, 3, device="cuda"))):
        d = dict(base)
        d.update(bad)
        with pytest.raises(RTError, match="INVALID_ARG"):
            Batch([base, d])
