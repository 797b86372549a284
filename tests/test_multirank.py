"""The multi-GPU path is replicas (no data-path collective): each rank runs
its own applications or its share of the excitations, and the job's timing is
the slowest rank's.  The host side of that -- the max over ranks, the
whole-job rate and the sharding of independent items -- runs here on two CPU
ranks over gloo, and so does a sharded computation (each rank's share of a
transducer's right-hand sides, by the oracle) checked against the whole job."""
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


def _rank_rhs(rank, world, port, out):
    """Rank's share of the excitations of a transducer: its right-hand sides
    by the oracle (no collective on the data path); the shards are gathered
    here only to check them."""
    import time

    import numpy as np
    import torch
    import torch.distributed as dist

    import bench
    from oracle import pmchwt, rayleigh
    from synth import scenes
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = scenes.two_sphere_scene(1)
        tr = scenes.bowl_transducer(seed=3, n_elem=6, R=4.0, aperture=3.0, piston_radius=0.3, gap=0.05)
        W = scenes.random_phase_weights(6, 5, seed=9)
        b, e = bench.shard(W.shape[0], rank, world)
        t0 = time.perf_counter()
        mine = [pmchwt.rhs(s, rayleigh.field(tr, W[r], s.k0, 2.0, 1.3)) for r in range(b, e)]
        dt = bench.max_over_ranks(time.perf_counter() - t0, world, device="cpu")
        parts = [None] * world
        dist.all_gather_object(parts, (b, e, [np.asarray(x) for x in mine]))
        out[rank] = (parts, dt)
    finally:
        dist.destroy_process_group()


def test_sharded_excitations_equal_the_whole_job():
    """Two replicas, each computing the right-hand sides of its contiguous
    share of five excitations with the oracle: together they cover every
    excitation once, and each equals the single-process result exactly."""
    import numpy as np

    from oracle import pmchwt, rayleigh
    from synth import scenes
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_rhs, args=(world, port, out), nprocs=world, join=True)
    parts, dt0 = out[0]
    assert out[1][1] == dt0 > 0
    s = scenes.two_sphere_scene(1)
    tr = scenes.bowl_transducer(seed=3, n_elem=6, R=4.0, aperture=3.0, piston_radius=0.3, gap=0.05)
    W = scenes.random_phase_weights(6, 5, seed=9)
    got = {}
    for b, e, xs in parts:
        for r, x in zip(range(b, e), xs):
            assert r not in got
            got[r] = x
    assert sorted(got) == list(range(5))
    for r in range(5):
        ref = pmchwt.rhs(s, rayleigh.field(tr, W[r], s.k0, 2.0, 1.3))
        assert np.array_equal(got[r], ref)

