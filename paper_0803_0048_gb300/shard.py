"""Batched solves over several GPUs: the items partitioned across ranks.

Every item of a batch (a7: a value set on a shared pattern, or a grid of its
own size) is an independent system, so N processes, one per GPU, can each
solve a share of the items in their own persistent launch (BatchSolve).
Nothing crosses GPUs while the items are solved; afterwards each item's
result (status, iterations, restart cycles, residual) is gathered on the host
of rank 0.  No device memory of one GPU is read by another.

The split balances estimated work.  An item's time in the batched kernel
grows with its rows (the arithmetic of its sweeps, mat-vecs and inner
products) and with the depth of its sweeps' dependency DAG (one barrier or
hand-off per level, twice per application), so the estimate is
rows x (forward depth + backward depth).  Items are assigned largest first,
each to the rank with the least estimated work so far (longest-processing-
time-first list scheduling, Graham 1969), ties to the lower rank; the result
is deterministic, so every rank computes the same partition without
communicating.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def item_cost(n: int, depth_lower: int, depth_upper: int) -> int:
    """Estimated work of one item: rows x (forward + backward DAG depth)."""
    if n < 0 or depth_lower < 0 or depth_upper < 0:
        raise ValueError("sizes and depths must be non-negative")
    return int(n) * (int(depth_lower) + int(depth_upper))


def partition(costs: Sequence[int], world: int) -> List[List[int]]:
    """Item indices per rank (each list ascending), largest cost first onto
    the least-loaded rank.  Every item lands on exactly one rank; a rank may
    receive none when there are fewer items than ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-int(costs[i]), i))
    load = [0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += int(costs[i])
    return [sorted(p) for p in parts]


def loads(costs: Sequence[int], parts: Sequence[Sequence[int]]) -> List[int]:
    """Estimated work per rank of a partition."""
    return [sum(int(costs[i]) for i in p) for p in parts]


def gather_results(local: Sequence[Tuple[int, tuple]], nitems: int, rank: int, world: int,
                   group=None) -> list:
    """Per-item results in item order on rank 0 (None on the other ranks).

    ``local`` holds (item index, result tuple) for the items this rank
    solved.  With world == 1 no process group is needed.  The results travel
    as host objects through torch.distributed (gloo or NCCL groups alike)."""
    if world == 1:
        merged = [None] * nitems
        for i, r in local:
            merged[i] = tuple(r)
        if any(r is None for r in merged):
            raise RuntimeError("items without a result")
        return merged
    import torch.distributed as dist
    payload = [(int(i), tuple(r)) for i, r in local]
    got = [None] * world if rank == 0 else None
    dist.gather_object(payload, got, dst=0, group=group)
    if rank != 0:
        return None
    merged = [None] * nitems
    for part in got:
        for i, r in part:
            if merged[i] is not None:
                raise RuntimeError(f"item {i} solved on two ranks")
            merged[i] = r
    missing = [i for i, r in enumerate(merged) if r is None]
    if missing:
        raise RuntimeError(f"items without a result: {missing[:8]}")
    return merged
