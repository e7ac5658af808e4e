"""Multi-process host logic on CPU (gloo, world size 2): shards partition the units and the
benchmark's timing reduction takes the max over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2511_03909_gb300.shard import reduce_max, shard_range


def test_shard_range_partitions():
    for total in (0, 1, 7, 256, 1000):
        for world in (1, 2, 3, 8):
            ranges = [shard_range(total, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == total
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        start, stop = shard_range(256, rank, world)
        mine = torch.arange(start, stop, dtype=torch.int64)
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, torch.tensor([mine.numel()]))
        got = [torch.zeros(int(s.item()), dtype=torch.int64) for s in sizes]
        # gloo all_gather needs equal sizes: pad to the largest
        m = max(int(s.item()) for s in sizes)
        pad = torch.full((m,), -1, dtype=torch.int64)
        pad[: mine.numel()] = mine
        outs = [torch.zeros(m, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(outs, pad)
        allu = torch.cat([o[o >= 0] for o in outs])
        ok = bool(torch.equal(torch.sort(allu).values, torch.arange(256)))
        t = reduce_max(1.5 + rank)
        q.put((rank, ok, t))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_sharding_and_max():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert all(ok for _, ok, _ in res)
    assert all(t == 2.5 for _, _, t in res)
