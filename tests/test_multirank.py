"""The benchmark's multi-rank path on CPU: two gloo ranks, as torchrun would
launch them.  Each rank gets its own disjoint seeds (weak scaling, no data
exchange) and the reported time is the maximum over ranks."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    seeds = list(bench.rank_seeds(rank, 8))
    t = bench.max_over_ranks(1.5 + rank, dist, "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    out.put((rank, seeds, t, gathered))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert res[0][1] == list(range(0, 8)) and res[1][1] == list(range(8, 16))
    assert all(r[2] == 2.5 for r in res)  # the slowest rank's time
    allseeds = res[0][3][0] + res[0][3][1]
    assert sorted(allseeds) == list(range(16))
