"""Multi-GPU host logic (replicas, no data-path collective) on CPU with gloo, world size 2."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

from paper_2402_01205_gb300.replicas import shard_balanced, shard_round_robin  # noqa: E402


def test_shards_are_disjoint_and_complete():
    sizes = [5, 1, 9, 3, 3, 7, 2, 8, 6, 4, 1]
    for world in (1, 2, 3, 4):
        rr = [shard_round_robin(len(sizes), r, world) for r in range(world)]
        bal = [shard_balanced(sizes, r, world) for r in range(world)]
        for parts in (rr, bal):
            flat = sorted(i for p in parts for i in p)
            assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in bal]
        assert max(loads) - min(loads) <= max(sizes)
    with pytest.raises(ValueError):
        shard_round_robin(3, 2, 2)


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2402_01205_gb300.replicas import max_over_ranks, shard_balanced, sum_over_ranks
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    sizes = [10, 20, 30, 40, 50]
    mine = shard_balanced(sizes, rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    elapsed = 1.0 + rank  # per-rank time
    mx = max_over_ranks(elapsed)
    tot = sum_over_ranks(sum(sizes[i] for i in mine))
    q.put((rank, got, mx, tot))
    dist.destroy_process_group()


def test_two_rank_gloo_replicas():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, mx, tot in out:
        assert sorted(got[0] + got[1]) == [0, 1, 2, 3, 4]
        assert mx == 2.0          # max over ranks of (1 + rank)
        assert tot == 150.0       # every cluster counted once
