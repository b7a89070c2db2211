"""The N > 1 path of bench.py on CPU: two gloo ranks (views split with no
exchange, the slowest rank's time taken with a MAX all-reduce)."""
import os
import socket
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    views = bench.shard_views(32, rank, world)
    shards = [None] * world
    dist.all_gather_object(shards, views)
    slowest = bench.max_over_ranks(1.0 + 2.5 * rank, world)
    dist.barrier()
    if rank == 0:
        out.put((shards, slowest))
    dist.destroy_process_group()


def test_two_gloo_ranks_split_views_and_take_the_slowest_time():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_rank_main, args=(2, port, q), nprocs=2, join=True, start_method="spawn")
    shards, slowest = q.get()
    flat = sorted(v for s in shards for v in s)
    assert flat == list(range(32))                        # every view once, no exchange needed
    assert len(shards[0]) == len(shards[1]) == 16         # weak scaling: the same work per rank
    assert slowest == 3.5


def test_shard_views_covers_views_for_any_rank_count():
    sys.path.insert(0, ROOT)
    import bench
    for world in (1, 2, 3, 4, 8, 40):
        shards = [bench.shard_views(32, r, world) for r in range(world)]
        if world <= 32:
            assert sorted(v for s in shards for v in s) == list(range(32))
        else:
            assert all(len(s) == 1 for s in shards)       # more ranks than views: one view each


def test_timed_views_spread_over_the_whole_path():
    """A run shorter than the path times evenly spaced views from the first
    (aerial) to the last (street); a longer one repeats the path."""
    sys.path.insert(0, ROOT)
    import bench
    for steps in (2, 5, 20, 31):
        v = bench.spread_views(list(range(32)), steps)
        assert len(v) == steps and v[0] == 0 and v[-1] == 31
        assert all(b > a for a, b in zip(v, v[1:]))
        gaps = [b - a for a, b in zip(v, v[1:])]
        assert max(gaps) - min(gaps) <= 1
    assert bench.spread_views(list(range(32)), 32) == list(range(32))
    assert bench.spread_views(list(range(32)), 40) == list(range(32)) + list(range(8))
    assert bench.spread_views(list(range(32)), 1) == [0]
