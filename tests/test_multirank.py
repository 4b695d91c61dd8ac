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
