"""One text over several ranks (one GPU each): contiguous ranges of start
positions, and ordered concatenation of the per-rank results.

Rank r owns the starts [s0, s1) with s0 = floor(r*S/W), s1 = floor((r+1)*S/W),
S = n - m + 1 starts and W ranks, and reads the bytes [s0, s1 + m - 1): every
occurrence is found by exactly one rank, the one owning its start, so the
global sorted list is the ranks' lists in rank order, each shifted by its s0.
The only exchange is one count per rank (and, to collect the positions on
every rank, an all-gather of the padded position lists).
"""
from __future__ import annotations


def shard_bounds(n: int, m: int, world: int, rank: int):
    """(s0, s1, b1): owned starts [s0, s1) and bytes to read [s0, b1)."""
    starts = n - m + 1 if n >= m else 0
    s0 = starts * rank // world
    s1 = starts * (rank + 1) // world
    b1 = s1 + m - 1 if s1 > s0 else s0
    return s0, s1, b1


def offsets_from_counts(counts):
    out = [0]
    for c in counts:
        out.append(out[-1] + int(c))
    return out


def sharded_search(search_shard, n: int, pattern: bytes, group=None):
    """Run ``search_shard(s0, b1, pattern)`` (local positions, ascending, of
    the shard's bytes [s0, b1)) on this rank and return (global positions,
    count) with every rank's results merged in order (torch.distributed)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    m = len(pattern)
    s0, s1, b1 = shard_bounds(n, m, world, rank)
    local = search_shard(s0, b1, pattern) if s1 > s0 else torch.zeros(0, dtype=torch.int64)
    local = torch.as_tensor(local, dtype=torch.int64).cpu() + s0
    cnt = torch.tensor([local.numel()], dtype=torch.int64)
    counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, cnt, group=group)
    counts = [int(c.item()) for c in counts]
    width = max(max(counts), 1)
    padded = torch.full((width,), -1, dtype=torch.int64)
    padded[:local.numel()] = local
    parts = [torch.empty(width, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    merged = torch.cat([p[:c] for p, c in zip(parts, counts)])
    return merged, sum(counts)
