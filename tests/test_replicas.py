"""The N > 1 launch of the benchmark on CPU: world-size-2 gloo ranks.

A single system does not shard (row i reads arbitrary earlier rows), so more
GPUs run independent replicas of the same step with no data-path collective.
What the ranks share is host logic: the time reported is the slowest
replica's, and under torchrun the oracle arm runs on rank 0 alone while the
other ranks exit 0 without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, values, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            rank=rank, world_size=world)
    try:
        q.put((rank, bench.ranks_max(values[rank], torch.device("cpu"), world)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_ranks_max_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    # each value's maximum sits on a different rank
    values = [[119.25, 7.0, -3.0], [118.5, 9.5, -4.0]]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, values, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0] == got[1] == [119.25, 9.5, -3.0]


def test_ranks_max_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.ranks_max([1.5, 2], None, 1) == [1.5, 2.0]


def _env(**kw):
    env = dict(os.environ)
    env.update({"MASTER_ADDR": "127.0.0.1"}, **kw)
    return env


def test_reference_arm_idle_rank_exits_quietly():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True,
                       text=True, timeout=120, env=_env(RANK="1", LOCAL_RANK="1", WORLD_SIZE="2"))
    assert r.returncode == 0, r.stderr
    assert r.stdout == ""


def test_reference_arm_under_torchrun_two_ranks():
    """torchrun with two ranks: exactly one JSON line, from rank 0."""
    port = _free_port()
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", str(port), "bench.py", "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600, env=_env())
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2
    assert out["higher_is_better"] is False and out["value"] > 0
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["value"] == out["value"]
    assert out["cpu_baseline"]["host"]["nproc"] >= 1
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["d2h_bytes_per_step"] == 0
