"""Batched items across ranks (paper_0803_0048_gb300.shard): the partition and
the gather of per-item results, on CPU with world-size-2 gloo ranks.

* The partition covers every item exactly once, is deterministic, keeps
  each rank's list ascending, and balances the estimated work within the
  largest single item (list scheduling's bound).
* Two gloo ranks each "solve" their share (a stand-in result derived from
  the item index) and rank 0 receives every item's result in item order.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_0803_0048_gb300 import shard  # noqa: E402


def batched_like_costs():
    # 512 equal value sets on one 32^3 pattern and 64 grids of sides 16..40
    # (depths ~3 side per sweep, as on a 7-point grid)
    sides = [16 + (7 * g) % 25 for g in range(64)]
    costs = [shard.item_cost(32 ** 3, 3 * 32, 3 * 32)] * 512
    costs += [shard.item_cost(s ** 3, 3 * s, 3 * s) for s in sides]
    return costs


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_items_once_and_balances(world):
    costs = batched_like_costs()
    parts = shard.partition(costs, world)
    assert len(parts) == world
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))
    assert all(p == sorted(p) for p in parts)
    ld = shard.loads(costs, parts)
    assert max(ld) - min(ld) <= max(costs)
    assert sum(ld) == sum(costs)
    assert parts == shard.partition(costs, world)  # deterministic


def test_partition_edge_cases():
    assert shard.partition([], 3) == [[], [], []]
    assert shard.partition([5], 2) == [[0], []]
    assert shard.partition([1, 1, 1, 1], 2) == [[0, 2], [1, 3]]
    # the largest item goes first, to rank 0; then the least-loaded rank
    assert shard.partition([1, 10, 1, 1], 2) == [[1], [0, 2, 3]]
    with pytest.raises(ValueError):
        shard.partition([1], 0)
    with pytest.raises(ValueError):
        shard.item_cost(-1, 2, 2)


def test_gather_single_rank():
    res = shard.gather_results([(1, (0, 5)), (0, (0, 4))], 2, 0, 1)
    assert res == [(0, 4), (0, 5)]
    with pytest.raises(RuntimeError):
        shard.gather_results([(1, (0, 5))], 2, 0, 1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_0803_0048_gb300 import shard as S
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            rank=rank, world_size=world)
    try:
        costs = batched_like_costs()
        parts = S.partition(costs, world)
        mine = parts[rank]
        # stand-in solve: status 0, iterations and residual from the index
        local = [(i, (0, 10 + i % 17, 1, 1e-9 * (i + 1))) for i in mine]
        merged = S.gather_results(local, len(costs), rank, world)
        q.put((rank, len(mine), merged))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_gather_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {r: (cnt, merged) for r, cnt, merged in (q.get(timeout=120) for _ in procs)}
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n = len(batched_like_costs())
    assert got[0][0] + got[1][0] == n and got[0][0] > 0 and got[1][0] > 0
    assert got[1][1] is None
    assert got[0][1] == [(0, 10 + i % 17, 1, 1e-9 * (i + 1)) for i in range(n)]
