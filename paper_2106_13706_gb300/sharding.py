"""Sharding of one exact ddKS problem, or of one permutation test, across
processes (one GPU each).

Every pooled point is an origin and origins are independent (Sec. 2.1), so a
problem splits into contiguous origin ranges; each rank runs
ddks_distance_range on its range and the shards combine with one exact
integer reduction: the largest numerator, then the lowest origin reaching it
(the library's arg-max convention).  No collective is needed on the data path;
the merge exchanges three integers per rank.

A permutation test (Sec. 4.2) splits by relabelling instead: relabelling b
depends only on the seed and b, so each rank runs its range [b_begin, b_end)
with ddks_permutation_test_range and the ranks add their counts of
num_b >= num_obs; p = (1 + total) / (1 + B).
"""
from __future__ import annotations


def shard_range(n_origins: int, world: int, rank: int):
    """Contiguous [begin, end) of origins for this rank (sizes differ by at most one)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    q, r = divmod(n_origins, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def merge_results(parts):
    """Combine per-shard results (dicts with num_max, argmax_origin, argmax_orthant,
    denom) into the result of the whole problem."""
    parts = [p for p in parts if p["argmax_origin"] >= 0]
    if not parts:
        raise ValueError("no non-empty shard")
    best = max(p["num_max"] for p in parts)
    winner = min((p for p in parts if p["num_max"] == best), key=lambda p: p["argmax_origin"])
    denom = parts[0]["denom"]
    return dict(num_max=best, denom=denom, D=best / denom, argmax_origin=winner["argmax_origin"],
                argmax_orthant=winner["argmax_orthant"])


def all_merge(result, group=None):
    """merge_results across the ranks of a torch.distributed group (any backend)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    t = torch.tensor([result["num_max"], result["argmax_origin"], result["argmax_orthant"],
                      result["denom"]], dtype=torch.int64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    out = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    parts = [dict(num_max=int(o[0]), argmax_origin=int(o[1]), argmax_orthant=int(o[2]),
                  denom=int(o[3])) for o in out]
    return merge_results(parts)


def merge_perm_counts(count_ge_parts, B):
    """p-value of a permutation test from the shards' counts of num_b >= num_obs."""
    if B < 0 or any(c < 0 for c in count_ge_parts):
        raise ValueError("bad counts")
    return (1 + sum(count_ge_parts)) / (1 + B)


def all_merge_perm(count_ge, B, group=None):
    """merge_perm_counts across the ranks of a torch.distributed group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([int(count_ge)], dtype=torch.int64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return merge_perm_counts([int(t.item())], B)
