"""Sharding one advance across ranks (paper Sec. 2: directions sharded across devices, a
per-shard sum, then one reduction across shards).

The partition is the library's (rt_shard_plan, a host function, called here on the CPU): every
(source, ray) pair in exactly one shard, shard sizes within one pair, at most three
rt_advance_rays pieces per shard, no divisibility condition on N_Omega. Two CPU ranks on gloo
then march their planned pieces -- with the FP64 oracle standing in for the GPU kernel, which
takes the same pieces (source subset, ray range) -- and sum their partial fields with one
all_reduce, as sharding.advance_distributed does with NCCL on GPUs; the result must equal the
unsharded field.
"""
import os

import numpy as np
import pytest

WORLD = 2


@pytest.fixture(scope="module")
def lib():
    from paper_2511_09389_gb300 import build, _native
    build.build()
    return _native.load()


@pytest.mark.parametrize("n_src,rays,world", [(3, 64, 2), (1, 97, 2), (16, 3072, 8), (5, 7, 3), (2097, 4096, 6),
                                             (2, 3, 8), (0, 5, 2), (7, 1, 4)])
def test_plan_covers_every_pair_once_and_balances(lib, n_src, rays, world):
    from paper_2511_09389_gb300 import sharding
    seen = np.zeros((n_src, rays), np.int64)
    sizes = []
    for r in range(world):
        pieces = sharding.plan(n_src, rays, world, r)
        assert len(pieces) <= 3
        size = 0
        for s0, s1, r0, r1 in pieces:
            assert 0 <= s0 < s1 <= n_src and 0 <= r0 < r1 <= rays
            seen[s0:s1, r0:r1] += 1
            size += (s1 - s0) * (r1 - r0)
        sizes.append(size)
    assert np.all(seen == 1)
    assert max(sizes) - min(sizes) <= 1 and sum(sizes) == n_src * rays


def test_plan_rejects_bad_arguments(lib):
    from paper_2511_09389_gb300 import sharding
    from paper_2511_09389_gb300._native import RTError
    for args in ((-1, 4, 2, 0), (3, 0, 2, 0), (3, 4, 0, 0), (3, 4, 2, 2), (3, 4, 2, -1)):
        with pytest.raises(RTError, match="INVALID_ARG"):
            sharding.plan(*args)


def _problem(n_src):
    from paper_2511_09389_gb300 import inputs
    return inputs.random_small(300 + n_src, shape=(10, 9, 11), n_freq=2, n_src=n_src, num_rays=64, horizon=8.0)


def _worker(rank, port, n_src, out_path):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2511_09389_gb300 import sharding

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    p = _problem(n_src)
    ns = oracle.num_substeps(p.step_size, 1.0, p.time_step)
    F = np.zeros_like(p.j, dtype=np.float64)
    for s0, s1, r0, r1 in sharding.plan(len(p.sources), p.num_rays, WORLD, rank):
        F += oracle.advance(p.j, p.kappa, p.sources[s0:s1], p.num_rays, p.step_size, ns, ray_range=(r0, r1))
    t = torch.from_numpy(F)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out_path, t.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("n_src", [3, 1, 4])
def test_two_rank_shards_reduce_to_the_whole(lib, tmp_path, n_src):
    """3 sources: a shard boundary inside a source's rays; 1 source: the rays split; 4 sources:
    whole sources per shard."""
    import socket

    import torch.multiprocessing as mp

    import oracle

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "F.npy")
    mp.start_processes(_worker, args=(port, n_src, out), nprocs=WORLD, start_method="spawn", join=True)
    F = np.load(out)
    p = _problem(n_src)
    R = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size,
                       oracle.num_substeps(p.step_size, 1.0, p.time_step))
    np.testing.assert_allclose(F, R, rtol=1e-12, atol=1e-13 * np.abs(R).max())
