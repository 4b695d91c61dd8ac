"""Host-side logic of the multi-GPU benchmark path, on CPU with gloo ranks.

Every rank integrates its own seeded domain (independent problems: weak
scaling, no data-path collective); the only collective is the max over ranks
of the measured time, which every rank then holds."""

import os
import socket

import numpy as np
import pytest
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
    from synth.fields import WORKLOADS, mechanism_for

    w = WORKLOADS["batched"]
    mech = mechanism_for(w)
    U = bench.batched_field(w, rank, n_cells=4096)
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



class _CpuTransport:
    """The ghost-row transport stencil and SSP-RK3 stages on CPU tensors, the
    same per-entry arithmetic on every slice and on the whole domain, so the
    comparison below isolates the domain decomposition and halo protocol."""

    def diffusion(self, Xext, D, dx):
        lap = (Xext[:-2] - 2.0 * Xext[1:-1]) + Xext[2:]
        return D * (lap / (dx * dx))

    def stage(self, stage, U1, Xext, S, sigma, out, D, dx, k):
        xk = Xext[1:-1] + k * (self.diffusion(Xext, D, dx) + sigma * S)
        if stage == 0:
            r = xk
        elif stage == 1:
            r = 0.75 * U1 + 0.25 * xk
        else:
            r = U1 / 3.0 + (2.0 / 3.0) * xk
        out.copy_(r)

    def empty_like(self, t):
        return torch.empty_like(t)


def _react(U, Tn):
    """A pointwise stand-in for the reaction sub-step (the decomposition does
    not touch it: each point is integrated on its own)."""
    U.add_(1e-7 * (Tn + 1e3 * torch.tanh(U)))


def _split_run(rank, world, U_all, nsteps, dt=1e-7, D=1e-4):
    import bench
    from paper_1712_00953_gb300 import halo_exchange, simpler_split_step_phases

    npts = U_all.shape[0]
    lo, hi = bench.shard_range(npts, rank, world)
    ext = torch.zeros(hi - lo + 2, U_all.shape[1], dtype=torch.float64)
    ext[1:-1] = torch.from_numpy(U_all[lo:hi])
    exchanges = 0
    for _ in range(nsteps):
        for x in simpler_split_step_phases(_react, _CpuTransport(), ext, dt, D, 1e-2 / npts):
            halo_exchange(x, rank, world)
            exchanges += 1
    return ext[1:-1].numpy().copy(), exchanges


def _halo_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    U_all = np.random.default_rng(5).normal(size=(37, 6)) * 100.0 + 1000.0
    out[rank] = _split_run(rank, world, U_all, 3)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_halo_sharded_split_steps_equal_single_rank_bitwise(world):
    """The 1-D domain (37 points, a ragged split) cut into contiguous slices
    over gloo ranks, one ghost row per side exchanged before each of the four
    transport evaluations of a Simpler split step: three split steps give the
    single-rank result bit for bit, with four exchanges per step."""
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_halo_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    U_all = np.random.default_rng(5).normal(size=(37, 6)) * 100.0 + 1000.0
    whole, n_ex = _split_run(0, 1, U_all, 3)
    got = np.concatenate([out[r][0] for r in range(world)], axis=0)
    assert all(out[r][1] == 12 for r in range(world)) and n_ex == 12
    assert not np.array_equal(whole, U_all)  # the steps did change the state
    np.testing.assert_array_equal(got, whole)
