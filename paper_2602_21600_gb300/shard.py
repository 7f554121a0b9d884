"""Database sharding over ranks: each rank holds one contiguous shard of the
base set with its own index, searches it, and the ranks exchange their
per-query top-k lists (one all-gather of k (distance, id) pairs per query
and rank) and merge them with ``aqr_merge_topk``.

The paper has no sharding: a shard's graph is an HNSW index of its own
points, so results differ from one graph over the whole set.  The merge
keeps Alg. 2's final ranking (distance, then id) over global ids.
"""

from __future__ import annotations


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Ids [lo, hi) of shard ``rank`` of ``world`` near-equal contiguous shards of n."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need 0 <= rank < world and n >= 0")
    return n * rank // world, n * (rank + 1) // world


def shard_offsets(n: int, world: int) -> list[int]:
    """Global id of the first point of every shard."""
    return [shard_range(n, r, world)[0] for r in range(world)]


def gather_lists(ids, dists, group=None):
    """All-gather of every rank's [n, k] result lists into [S, n, k] tensors
    (rank order), on whatever device the tensors live (NCCL for CUDA
    tensors, gloo for CPU ones)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return ids[None], dists[None]
    world = dist.get_world_size(group)
    gi = [torch.empty_like(ids) for _ in range(world)]
    gd = [torch.empty_like(dists) for _ in range(world)]
    dist.all_gather(gi, ids.contiguous(), group=group)
    dist.all_gather(gd, dists.contiguous(), group=group)
    return torch.stack(gi), torch.stack(gd)


def sharded_search(ctx, q, k: int, ef: int, n_total: int, group=None, stream=None):
    """Search this rank's shard with ``ctx`` (its index holds the points
    ``shard_range(n_total, rank, world)``), exchange the lists and merge:
    returns global ids and distances [n, k] on every rank."""
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
    ids, dists = ctx.search(q, k, ef, stream=stream)
    gi, gd = gather_lists(ids, dists, group)
    return ctx.merge_topk(gd, gi, shard_offsets(n_total, world), stream=stream)
