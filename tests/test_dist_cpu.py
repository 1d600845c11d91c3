"""The multi-rank host logic on CPU: two gloo ranks shard a batch of problems
(every problem on exactly one rank) and combine timings by a maximum."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_0803_1975_gb300.dist import max_over_ranks, shard


def test_shard_partitions():
    for count in (0, 1, 5, 4096, 4097):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                s = shard(count, r, world)
                seen.extend(s)
                assert abs(len(s) - count / world) < 1
            assert seen == list(range(count))
    with pytest.raises(ValueError):
        shard(4, 2, 2)


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
    count = 4096
    mine = shard(count, rank, world)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([len(mine)], dtype=torch.int64))
    firsts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(firsts, torch.tensor([mine.start], dtype=torch.int64))
    m = max_over_ranks(1.5 + rank)
    dist.destroy_process_group()
    q.put((rank, [int(x) for x in sizes], [int(x) for x in firsts], m))


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, sizes, firsts, m in out:
        assert sum(sizes) == 4096 and firsts == [0, sizes[0]]
        assert m == 2.5
    assert max_over_ranks(3.25) == 3.25        # no process group in this process
