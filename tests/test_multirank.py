"""Host-side logic of the multi-GPU benchmark path, on CPU with gloo ranks.

Every rank integrates its own seeded domain (independent problems: weak
scaling, no data-path collective); the only collective is the max over ranks
of the measured time, which every rank then holds."""

import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    w, mech, U = bench.build_inputs(rank)
    t = bench.max_over_ranks(0.5 + rank, dist, "cpu")
    out[rank] = (float(U[:, 0].sum()), float(mech.arrh.sum()), t)  # Y_1 depends on the seed
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_host_logic():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    (f0, m0, t0), (f1, m1, t1) = out[0], out[1]
    assert m0 == m1  # same mechanism on every rank
    assert f0 != f1  # independent seeded domains
    assert t0 == t1 == 1.5  # every rank holds the slowest rank's time


def _shard_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    n = 1001
    lo, hi = bench.shard_range(n, rank, world)
    rng = np.random.default_rng(0)
    st_all = np.stack([rng.integers(1, 50, n), rng.integers(0, 5, n), rng.integers(3, 200, n),
                       (rng.random(n) < 0.01).astype(int)], axis=1)
    out[rank] = ((lo, hi), bench.reduce_stats(st_all[lo:hi], dist, "cpu"), bench.reduce_stats(st_all, None, "cpu"))
    dist.barrier()
    dist.destroy_process_group()


def test_three_gloo_ranks_shard_independent_cells():
    """Sharding the batched cells: contiguous slices cover every cell once, and
    the all-reduced statistics equal those of the whole set."""
    world = 3
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_shard_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    ranges = sorted(out[r][0] for r in range(world))
    assert ranges[0][0] == 0 and ranges[-1][1] == 1001
    assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    assert max(h - l for l, h in ranges) - min(h - l for l, h in ranges) <= 1
    whole = out[0][2]
    for r in range(world):
        assert out[r][1] == whole

