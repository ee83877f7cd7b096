"""One advance split across ranks (Sec. 2: directions sharded across devices, a per-device sum,
then one reduction across devices).

Each rank marches its shard of the (source, ray) pairs -- planned by the library's
rt_shard_plan, balanced to one pair, with no divisibility condition on N_Omega -- into a partial
field on its own GPU; one all-reduce (sum) over the ranks' partial fields gives every rank the
whole field. j and kappa are replicated (read-only); the partial fields are the only data that
moves between devices.
"""
from __future__ import annotations

import ctypes

from . import _native
from ._native import check


def plan(num_sources: int, num_rays: int, n_shards: int, shard: int):
    """The pieces (source_begin, source_end, ray_begin, ray_end) of one shard (rt_shard_plan)."""
    lib = _native.load()
    buf = (ctypes.c_int * 12)()
    n = ctypes.c_int()
    check(lib.rt_shard_plan(int(num_sources), int(num_rays), int(n_shards), int(shard), buf, ctypes.byref(n)))
    return [tuple(buf[4 * i:4 * i + 4]) for i in range(n.value)]


def advance_shard(grid, j, kappa, sources, num_rays: int, step_size: float, radiation_velocity: float,
                  time_step: float, rank: int, world: int, out, stream=None):
    """This rank's partial field: its pieces marched with rt_advance_rays into `out` (overwritten;
    zero when the shard is empty)."""
    pieces = plan(sources.shape[0], num_rays, world, rank)
    if not pieces:
        out.zero_()
        return out
    for i, (s0, s1, r0, r1) in enumerate(pieces):
        grid.advance(j, kappa, sources[s0:s1], num_rays, step_size, radiation_velocity, time_step, out=out,
                     accumulate=i > 0, ray_range=(r0, r1), stream=stream)
    return out


def advance_distributed(grid, j, kappa, sources, num_rays: int, step_size: float, radiation_velocity: float,
                        time_step: float, out, group=None):
    """The whole field on every rank of the default (or given) process group: this rank's shard,
    then one all-reduce (sum) of the partial fields."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    advance_shard(grid, j, kappa, sources, num_rays, step_size, radiation_velocity, time_step, rank, world, out)
    dist.all_reduce(out, op=dist.ReduceOp.SUM, group=group)
    return out
