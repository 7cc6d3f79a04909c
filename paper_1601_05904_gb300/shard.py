"""Query-sharded AIDW over several GPUs, one process per GPU.

Every query of Eq. 1 is computed independently given all data points (the
paper's one-thread-per-query decomposition, Sec. 4.2), so one query set
splits over G GPUs with no exchange on the data path: each process builds
its own grid from a replica of the data points, interpolates one contiguous
slice of the queries (``aidw_shard_range`` / ``aidw_interpolate_shard`` of
the C ABI) and writes that slice of the output.  Bringing the slices
together is an optional all-gather of the results, after the computation.

This module only marshals: the slicing rule is the library's
``aidw_shard_range`` and all arithmetic runs in ``libaidw.so``.
"""
from __future__ import annotations

from . import binding


def slices(n_query: int, world: int) -> list[tuple[int, int]]:
    """[begin, end) of every shard, in shard order (the library's rule)."""
    return [binding.aidw_shard_range(n_query, r, world) for r in range(world)]


def gather_slices(full_local, n_query: int, group=None):
    """All-gathers the shards' slices into one full-length tensor on every rank.

    ``full_local`` is a full-length tensor [n_query] in which this rank has
    written its own slice; the result holds every rank's slice in place.
    Works with any torch.distributed backend whose device matches the tensor
    (gloo on CPU tensors, NCCL on CUDA tensors)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    sl = slices(n_query, world)
    width = max(e - b for b, e in sl) if sl else 0
    b, e = sl[rank]
    send = torch.zeros(width, dtype=full_local.dtype, device=full_local.device)
    send[: e - b] = full_local[b:e]
    recv = [torch.empty_like(send) for _ in range(world)]
    dist.all_gather(recv, send, group=group)
    return torch.cat([recv[r][: e_r - b_r] for r, (b_r, e_r) in enumerate(sl)])


def interpolate_sharded(x, y, z, qx, qy, params: binding.Params | None = None, group=None,
                        gather: bool = True, stream=None):
    """AIDW of the full query set (qx, qy) split over the ranks of ``group``.

    Every rank passes the same data (x, y, z) and queries (qx, qy) as CUDA
    tensors on its own GPU.  The rank builds a grid from the data,
    interpolates its slice and returns either the full prediction vector
    (``gather=True``: the slices of all ranks, all-gathered) or its
    full-length local vector with only its own slice written (the other
    elements are NaN).  Without torch.distributed initialised, or with one
    rank, this is ``aidw_interpolate`` of the whole set."""
    import torch.distributed as dist
    world, rank = 1, 0
    if dist.is_available() and dist.is_initialized():
        world, rank = dist.get_world_size(group), dist.get_rank(group)
    g = binding.aidw_grid_build(x, y, z, params, stream)
    try:
        out, _ = binding.aidw_interpolate_shard(g, qx, qy, rank, world, params, stream=stream)
    finally:
        g.destroy()
    if gather and world > 1:
        out = gather_slices(out, qx.numel(), group)
    return out
