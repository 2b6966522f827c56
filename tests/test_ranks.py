"""bench.py's multi-GPU form on CPU: world size 2 over gloo.  Ranks take
disjoint slices (replicas, weak scaling), the timed region is the max over
ranks, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ids = bench.shard_ids(rank, world, 4)
    slow = bench.max_over_ranks(10.0 * (rank + 1), world, "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, ids)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ids, slow, gathered))


def test_two_ranks_shard_and_take_the_slowest():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ids, slow, gathered in out:
        assert slow == 20.0
        assert ids == list(range(4 * rank, 4 * rank + 4))
        assert not set(gathered[0]) & set(gathered[1])


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup, gpus = 1, 0, 2
    assert bench.run_reference(Args(), rank=1, world=2) == 0
    assert capsys.readouterr().out == ""
