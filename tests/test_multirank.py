"""The multi-GPU path is replicas (no data-path collective): each rank runs
its own applications or its share of the excitations, and the job's timing is
the slowest rank's.  The host side of that -- the max over ranks, the
whole-job rate and the sharding of independent items -- runs here on two CPU
ranks over gloo."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.5 + rank, world, device="cpu")   # rank 1 is the slow one
        b, e = bench.shard(7, rank, world)
        out[rank] = (t, bench.job_rate(100.0, world, t), b, e)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 2.5           # every rank sees the slowest time
    assert out[0][1] == pytest.approx(200.0 / 2.5)  # all ranks' units over that time
    assert (out[0][2], out[0][3], out[1][2], out[1][3]) == (0, 4, 4, 7)


@pytest.mark.parametrize("n,world", [(0, 3), (5, 1), (10, 4), (3, 8)])
def test_shards_cover_every_item_once(n, world):
    import bench
    parts = [bench.shard(n, r, world) for r in range(world)]
    assert parts[0][0] == 0 and parts[-1][1] == n
    assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
    sizes = [e - b for b, e in parts]
    assert max(sizes) - min(sizes) <= 1
