"""Sharding of the march across ranks (paper Sec. 2: directions sharded across devices, a
per-shard sum, then one reduction across shards), run as two CPU ranks with the gloo backend.

Each rank marches its part of the work with the FP64 oracle and the partial fields are summed
with one all_reduce; the result must equal the unsharded field. Sharding by directions needs
N_Omega divisible by the rank count in the paper; splitting the (source, direction) space, as
here by sources too, removes that constraint.
"""
import os

import numpy as np
import pytest

WORLD = 2


def _worker(rank, port, mode, out_path):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2511_09389_gb300 import inputs

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    p = inputs.random_small(300, shape=(10, 9, 11), n_freq=2, n_src=3, num_rays=64, horizon=8.0)
    ns = oracle.num_substeps(p.step_size, 1.0, p.time_step)
    if mode == "directions":
        per = p.num_rays // WORLD
        F = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns,
                           ray_range=(rank * per, (rank + 1) * per))
    else:  # sources, uneven split
        src = p.sources[:1] if rank == 0 else p.sources[1:]
        F = oracle.advance(p.j, p.kappa, src, p.num_rays, p.step_size, ns)
    t = torch.from_numpy(F)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out_path, t.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["directions", "sources"])
def test_two_rank_shards_reduce_to_the_whole(tmp_path, mode):
    import socket

    import torch.multiprocessing as mp

    import oracle
    from paper_2511_09389_gb300 import inputs

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "F.npy")
    mp.start_processes(_worker, args=(port, mode, out), nprocs=WORLD, start_method="spawn", join=True)
    F = np.load(out)
    p = inputs.random_small(300, shape=(10, 9, 11), n_freq=2, n_src=3, num_rays=64, horizon=8.0)
    R = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size,
                       oracle.num_substeps(p.step_size, 1.0, p.time_step))
    np.testing.assert_allclose(F, R, rtol=1e-12, atol=1e-13 * np.abs(R).max())
