"""Rays sharded over several GPUs (one process per GPU).

Rays are independent (Sec. III.B: every ray is traced on its own), so a batch
splits into contiguous ray ranges, one per rank; every rank holds a replica of
the scene and its BVH, traces its own range through the library, and writes
its hits in place.  No step of the path exchanges data: the only collective is
the optional gather that hands every rank the whole hit array.

Used under torch.distributed (NCCL for GPUs; any backend for the host-side
logic).  The tracing itself stays in librtbvh on each rank's GPU.
"""
from __future__ import annotations


def ray_range(n: int, rank: int, world: int):
    """The contiguous range [lo, hi) of n rays that `rank` of `world` traces:
    balanced (sizes differ by at most one, larger ranges first), disjoint,
    covering [0, n) in rank order."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad rank %r / world %r / n %r" % (rank, world, n))
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def gather_ranges(local, n: int, group=None):
    """All-gather of per-rank row ranges (ray_range order) into the full
    [n, ...] tensor on every rank.  `local` holds this rank's rows; ranges of
    unequal size are padded to the largest for the collective and cut back."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    lo, hi = ray_range(n, rank, world)
    if local.shape[0] != hi - lo:
        raise ValueError("rank %d holds %d rows, its range has %d" % (rank, local.shape[0], hi - lo))
    width = ray_range(n, 0, world)[1]  # the largest range
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: hi - lo] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    out = [parts[k][: ray_range(n, k, world)[1] - ray_range(n, k, world)[0]] for k in range(world)]
    return torch.cat(out, 0)


def trace_closest_sharded(scene, rays, group=None, gather=True, stream=None, **trace_kw):
    """Closest hits of `rays` (the whole batch, on this rank's GPU) with the
    rays split over the ranks of `group`: this rank traces its range with
    rt_trace_closest; with gather, every rank returns all n hits (one
    all-gather), else only its own range and (lo, hi)."""
    import torch.distributed as dist
    from . import rtbvh
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    n = rays.shape[0]
    lo, hi = ray_range(n, rank, world)
    hits = rtbvh.rt_trace_closest(scene, rays[lo:hi], stream=stream, **trace_kw)
    if not gather:
        return hits, (lo, hi)
    return gather_ranges(hits, n, group)
