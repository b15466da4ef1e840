"""Multi-rank host logic on CPU (gloo, world size 2): plane ranges partition
the planes, and the max over ranks that the benchmark's timing uses."""

import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1503_07998_gb300 import shard


def test_plane_ranges_partition():
    for P in (0, 1, 5, 512, 1023):
        for world in (1, 2, 3, 8):
            ranges = [shard.plane_range(P, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == P
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    assert shard.volumes_of_rank(5, 1, 2) == [1, 3]
    with pytest.raises(ValueError):
        shard.plane_range(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = shard.plane_range(7, rank, world)
        t = torch.tensor([lo, hi], dtype=torch.int64)
        parts = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(parts, t)
        out[rank] = (shard.max_over_ranks(10.0 * (rank + 1)), [p.tolist() for p in parts])
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_planes_and_take_the_max_time():
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        mx, parts = res[rank]
        assert mx == 20.0
        assert parts == [[0, 4], [4, 7]]
