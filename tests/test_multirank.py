"""Multi-rank logic of bench.py on CPU (gloo, world size 2).

On the GPU every rank solves its own problems ("replicas only": a single solve
is not sharded), the job time is the slowest rank's, and the batched workload
is split by a size-balanced greedy assignment with no collective on the data path.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as w
    probs = w.c5_batch()
    mine = bench.shard(probs, rank, world)
    slowest = bench.max_over_ranks(10.0 + rank, world)
    dist.barrier()
    q.put((rank, [p.name for p in mine], slowest))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    names0, names1 = res[0][1], res[1][1]
    import workloads as w
    allnames = [p.name for p in w.c5_batch()]
    assert not set(names0) & set(names1)
    assert sorted(names0 + names1) == sorted(allnames)
    assert res[0][2] == res[1][2] == 11.0


def test_batched_split_is_balanced_and_complete():
    # every problem on exactly one rank, and the ranks' node counts within a few
    # per cent of each other (largest-first greedy on the 470x volume spread)
    import bench
    import workloads as w
    probs = w.c5_batch()
    total = sum(p.points for p in probs)
    for world in (2, 4, 8):
        parts = [bench.shard(probs, r, world) for r in range(world)]
        names = sorted(p.name for part in parts for p in part)
        assert names == sorted(p.name for p in probs)
        loads = [sum(p.points for p in part) for part in parts]
        assert max(loads) <= 1.05 * total / world, (world, loads)
