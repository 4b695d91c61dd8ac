"""Benchmark: Simpler balanced split steps of the 1-D reaction-diffusion workload.

One bench step = one Simpler balanced split step (Eq. simpler_balanced) of the
1-D reaction-diffusion system: 2048 points on 1 cm, a 30-species /
150-reaction synthetic mechanism (4 third-body, 2 Troe falloff reactions),
tanh temperature front 300 -> 2000 K, dt = 1e-7 s, ROK4E with M = 4,
rtol 1e-6, atol 1e-10: transport T(U_n), the per-cell ROK4E reaction
sub-step with the constant source T(U_n), and the SSP-RK3 transport
correction over dt/2.  Metric: cell-steps/s = points x split steps / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank integrates its own independent domain
(seeded per rank): weak scaling, no data-path collective.  ``--impl reference``
times the FP64 numpy oracle on the host cores on a bounded sample of the same
workload (rank 0 only).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "flame1d"
D_DIFF = 1.0e-4  # m^2/s
LENGTH = 1.0e-2  # m
P_ATM = 101325.0
L2_FLUSH_BYTES = 256 << 20
PREC = {"fp64": 0, "mixed": 1, "mixed-fp32jv": 2, "mixed-df": 3}


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


# ------------------------------------------------------------- work model
def flop_model(mech, M):
    """Algorithmic FP64 operation counts (flops, FMA = 2) of the kernels' units.

    Returns dict(rhs, rhs_exp, jvp, arnoldi, attempt) per unit.  Transcendentals
    are counted separately (rhs_exp) and converted with the measured cost of
    one FP64 exp in FMA-equivalents."""
    ns, nr = mech.n_species, mech.n_reactions
    N = ns + 1
    kind = np.asarray(mech.kind)
    n_tb = int((kind == 1).sum())
    n_troe = int((kind == 2).sum())
    nnz = 0
    for j in range(nr):
        net = {}
        for s, n in zip(mech.rxn_sp[j], mech.rxn_nu[j]):
            if s >= 0:
                net[s] = net.get(s, 0) + n
        nnz += sum(1 for v in net.values() if v != 0)
    rhs = ns * 40 + nr * 16 + 2 * nnz + (n_tb + n_troe) * 2 * ns + n_troe * 40 + 10
    rhs_exp = 2 * ns + nr + 7 * n_troe + 1
    jvp = ns * 25 + nr * 26 + 2 * nnz + (n_tb + n_troe) * (2 * ns + 4) + 10
    arnoldi = 3 * N + M * 5 * N + 8 * N * M * (M + 1) // 2
    attempt = 4 * N * (4 * M + 6) + 22 * N + (2 * M**3) // 3 + 8 * M * M
    return dict(rhs=rhs, rhs_exp=rhs_exp, jvp=jvp, arnoldi=arnoldi, attempt=attempt)


EXP_FLOPS = 20  # one FP64 exp counted as 10 operations (the table-driven method's count)


def algorithmic_flops(model, stats, M, exp_flops=EXP_FLOPS):
    """Total FP64 flops implied by per-cell stats (one exp = exp_flops)."""
    st = np.asarray(stats, dtype=np.int64).reshape(-1, 4)
    n_acc, n_rej, n_rhs = st[:, 0].sum(), st[:, 1].sum(), st[:, 2].sum()
    n_arn = np.maximum(st[:, 0], 1).sum()
    rhs_total = n_rhs * (model["rhs"] + exp_flops * model["rhs_exp"])
    return float(rhs_total + n_arn * (M * model["jvp"] + model["arnoldi"]) + (n_acc + n_rej) * model["attempt"])


def shard_range(n, rank, world):
    """Contiguous, near-equal slice [lo, hi) of n independent cells for one rank."""
    return n * rank // world, n * (rank + 1) // world


def reduce_stats(st, dist, device):
    """Totals over every rank's cells from per-cell statistics [n_local, 4]
    (accepted, rejected, RHS evaluations, status): summed accepted steps,
    attempts and RHS evaluations, the largest substep count, the number of
    failed cells and of cells (a sum and a max all-reduce); without ``dist``
    the local totals."""
    import torch

    st = np.asarray(st, dtype=np.int64).reshape(-1, 4)
    sums = torch.tensor([float(st[:, 0].sum()), float((st[:, 0] + st[:, 1]).sum()), float(st[:, 2].sum()),
                         float((st[:, 3] != 0).sum()), float(st.shape[0])], dtype=torch.float64, device=device)
    mx = torch.tensor([float(st[:, 0].max()) if st.shape[0] else 0.0], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(sums, op=dist.ReduceOp.SUM)
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    acc, a, r, f, c = (float(x) for x in sums.cpu())
    return {"accepted": acc, "attempts": a, "rhs": r, "failed_cells": int(f), "cells": int(c),
            "substeps_max": int(mx.item())}


def max_over_ranks(t, dist, device):
    """The slowest rank's time (every rank gets it); ``dist`` is None for one process."""
    if dist is None:
        return t
    import torch

    x = torch.tensor([t], device=device, dtype=torch.float64)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())


# -------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu_index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- arms
def build_inputs(rank):
    from synth.fields import WORKLOADS, field_tanh_front, mechanism_for

    w = WORKLOADS[WORKLOAD]
    mech = mechanism_for(w)
    _, U = field_tanh_front(w.n_cells, w.n_species, w.field_seed + 97 * rank)
    return w, mech, U


def stratified_cells(npts, n_cells, offset=0):
    """n_cells cell indices spread over the grid (golden-ratio sequence)."""
    return [int((offset + i) * 0.6180339887498949 * npts) % npts for i in range(n_cells)]


def cpu_oracle_sample(w, mech, U, cells):
    """Time the oracle's Simpler split step on a sample of cells: transport over
    the whole grid, the ROK4E reaction sub-step on the listed cells."""
    from oracle import splitting as osp
    from oracle.kinetics import Kinetics

    kin = Kinetics(mech)
    npts = U.shape[0]
    dx = LENGTH / npts
    n_cells = len(cells)
    t0 = time.perf_counter()
    _, _, _, U_react = osp.simpler_split_step_1d(kin, U, P_ATM, w.dt, D_DIFF, dx, w.rtol, w.atol, w.krylov_dim,
                                                 cells=cells)
    dt = time.perf_counter() - t0
    return n_cells / dt, dt, U_react


def _oracle_cell(task):
    """One cell's ROK4E reaction sub-step through the oracle (worker process)."""
    from oracle import rok4e
    from oracle.kinetics import Kinetics

    mech, u0, src, dt, rtol, atol, M = task
    f, jv_at = rok4e.reactor(Kinetics(mech), P_ATM, src)
    return rok4e.integrate(f, jv_at, u0, dt, rtol, atol, M)[0]


def cpu_oracle_sample_all_cores(w, mech, U, cells):
    """The same oracle sample spread over every host core (one process per core,
    spawned, so no CUDA state is inherited): the reaction sub-steps of the
    listed cells with the transport source T(U_n); cells/s and the core count."""
    import multiprocessing as mp

    from oracle import splitting as osp

    npts = U.shape[0]
    Tn = osp.diffusion_op(U, D_DIFF, LENGTH / npts)
    procs = max(1, min(os.cpu_count() or 1, len(cells)))
    tasks = [(mech, U[c], Tn[c], w.dt, w.rtol, w.atol, w.krylov_dim) for c in cells]
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_cell, tasks[:procs])  # start-up (imports) outside the timing
        t0 = time.perf_counter()
        pool.map(_oracle_cell, tasks, chunksize=1)
        dt = time.perf_counter() - t0
    return len(cells) / dt, procs, dt


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    w, mech, U = build_inputs(0)
    per_step = 1
    npts = U.shape[0]
    for k in range(args.warmup):
        cpu_oracle_sample(w, mech, U, stratified_cells(npts, per_step, 1000 + k))
    t_total = 0.0
    cells_total = 0
    for k in range(args.steps):
        _, dt, _ = cpu_oracle_sample(w, mech, U, stratified_cells(npts, per_step, k))
        t_total += dt
        cells_total += per_step
    value = cells_total / t_total
    line = {
        "impl": "reference", "metric": "cell-steps/s", "value": value, "unit": "cell-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "flame1d 1-D reaction-diffusion, 2048 points, 30 species / 150 reactions, "
                               "Simpler split steps of 1e-7 s, ROK4E M=4, rtol 1e-6, atol 1e-10",
                   "oracle_sample": f"{per_step} cell(s) per step through the FP64 numpy oracle"},
        "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} cell per step (golden-ratio sequence over the grid) x "
                                   f"{args.steps} steps, one split step of the initial field each"},
        "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_plain(args):
    """Untimed split steps of the workload (the small case used for ncu captures)."""
    import torch

    import paper_1712_00953_gb300 as rk

    w, mech, U0 = build_inputs(0)
    m = rk.mech_load(mech)
    U = torch.tensor(U0, device="cuda")
    hc = torch.zeros(U.shape[0], dtype=torch.float64, device="cuda")
    for _ in range(args.plain_steps):
        rk.simpler_split_step(m, U, w.dt, D_DIFF, LENGTH / U.shape[0], w.rtol, w.atol, w.krylov_dim, h_cell=hc,
                              opts=rk.Opts(lanes_per_cell=args.lanes, cells_per_block=args.cells_per_block,
                                           precision=PREC[args.precision], queue_order=args.queue_order, blocks_per_sm=args.blocks_per_sm))
    torch.cuda.synchronize()
    print(json.dumps({"plain_steps": args.plain_steps, "T_max": float(U[:, -1].max())}))
    return 0


def run_unit_costs(args):
    """Small launches for per-unit FP64 instruction accounting under ncu (one
    RHS, one J v and one integration launch over 4096 cells for the flame1d and
    batched mechanisms), then the arithmetic-unit probes."""
    import torch

    import paper_1712_00953_gb300 as rk
    from synth.fields import WORKLOADS, field_uniform, mechanism_for

    for name in ("flame1d", "batched"):
        w = WORKLOADS[name]
        mech = mechanism_for(w)
        m = rk.mech_load(mech)
        n = 4096
        U = torch.tensor(field_uniform(n, mech.n_species, 5, 1500.0, 2300.0), device="cuda")
        V = torch.randn_like(U)
        rk.chem_rhs(m, U, P_ATM)
        rk.chem_jvp(m, U, V, P_ATM, mode=0)
        st = torch.zeros(n, 4, dtype=torch.int32, device="cuda")
        Y = U.clone()
        rk.rok4e_integrate(m, Y, 1e-7, w.rtol, w.atol, 4, stats=st, opts=rk.Opts(cells_per_block=8))
        torch.cuda.synchronize()
        s = st.cpu().numpy()
        print(json.dumps({"unit_costs": name, "cells": n, "attempts": int((s[:, 0] + s[:, 1]).sum()),
                          "rhs": int(s[:, 2].sum()), "failed": int((s[:, 3] != 0).sum())}))
    if not args.skip_probes:
        names = ["fp64_fma", "fp32_fma", "fp64_exp", "cvt", "fp64_fma_1warp_per_sm", "fp64_fma_4warps_per_sm",
                 "fp64_warp_inst_1lane_4warps_per_sm", "df_fma"]
        print(json.dumps({"probes_ops_per_s": {nm: rk.probe_throughput(k) for k, nm in enumerate(names)}}))
    return 0


def run_batched(args, rank, world, local_rank):
    """The batched workload: 2^20 independent constant-pressure cells from a
    Gaussian random temperature field, one ROK4E integration of dt = 1e-6 s
    (M = 4) per step from the same initial field; cell-steps/s.  On N GPUs the
    2^20 cells are sharded contiguously over the ranks (strong scaling: the
    cells are independent, so no data moves between GPUs); the statistics are
    all-reduced and the time is the slowest rank's."""
    import torch

    import paper_1712_00953_gb300 as rk
    from synth.fields import WORKLOADS, initial_state, mechanism_for

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl", device_id=dev)
    w = WORKLOADS["batched"]
    mech = mechanism_for(w)
    U_all = initial_state(w)
    n_total = U_all.shape[0]
    lo, hi = shard_range(n_total, rank, world)
    U0 = torch.tensor(U_all[lo:hi], device=dev)
    del U_all
    n = U0.shape[0]
    m = rk.mech_load(mech)
    M = w.krylov_dim
    Y = torch.empty_like(U0)
    st = torch.zeros(n, 4, dtype=torch.int32, device=dev)
    ws = torch.empty(rk.rok4e_workspace_size(m, n, M), dtype=torch.uint8, device=dev)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for a in ev:
        a.record()
    o = rk.Opts(lanes_per_cell=args.lanes, cells_per_block=args.cells_per_block, blocks_per_sm=args.blocks_per_sm,
                precision=PREC[args.precision], events=ev)
    for _ in range(args.warmup):
        Y.copy_(U0)
        rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, M, opts=o, workspace=ws)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    kern = 0.0
    flops = 0.0
    model = flop_model(mech, M)
    for _ in range(args.steps):
        Y.copy_(U0)  # 2^20 x 54 doubles = 453 MB: larger than L2
        rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, M, opts=o, stats=st, workspace=ws)
        torch.cuda.synchronize()
        kern += ev[0].elapsed_time(ev[1]) * 1e-3
        flops += algorithmic_flops(model, st.cpu().numpy(), M)
    kern_max = max_over_ranks(kern, dist, dev)
    flops_all = flops
    tot = reduce_stats(st.cpu().numpy(), dist, dev)
    if dist:
        fl = torch.tensor([flops], dtype=torch.float64, device=dev)
        dist.all_reduce(fl, op=dist.ReduceOp.SUM)
        flops_all = float(fl.item())
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {"workload": "batched: 2^20 cells, 53 species / 325 reactions, one 1e-6 s ROK4E step, M=4",
            "precision": args.precision, "n_gpus": world, "scaling": "strong" if world > 1 else "weak",
            "cells_per_gpu": n, "cell_steps_per_s": n_total * args.steps / kern_max,
            "kernel_s_per_step": kern_max / args.steps,
            "roofline": {"bound": "alu", "achieved": flops_all / kern_max / 1e12 / world, "peak": 1.25,
                         "unit": "TFLOP/s per GPU", "frac": flops_all / kern_max / 1e12 / 1.25 / world},
            "substeps_mean": tot["accepted"] / tot["cells"], "substeps_max": tot["substeps_max"],
            "attempts_per_s": tot["attempts"] * args.steps / kern_max,
            "failed_cells": tot["failed_cells"]}
    print(json.dumps(line))
    return 0


def run_study(args, local_rank):
    """Efficiency study (Sec. 4.4's comparison on GPU): integrate 1024 cells of
    the batched workload's field (53 species / 325 reactions) over 1e-5 s in
    splitting intervals h_CFL in {1e-9 .. 1e-5} s, carrying each cell's step
    across intervals, with ROK4E M = 4, 6, 8 (analytic J v), ROK4E M = 4 with
    finite-difference J v, and the explicit Dormand-Prince 5(4) pair, all at
    rtol 1e-4, atol 1e-8.  Error: relative temperature error at 1e-5 s against
    a tight-tolerance reference (ROK4E M = 8, rtol 1e-10, atol 1e-14, checked
    against Dormand-Prince at the same tolerances).  One JSON line per case."""
    import torch

    import paper_1712_00953_gb300 as rk
    from synth.fields import WORKLOADS, initial_state, mechanism_for

    import dataclasses

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = WORKLOADS["batched"]
    if args.study_kcap > 0:  # a stiffer variant of the mechanism (larger cap on k C)
        w = dataclasses.replace(w, k_cap=args.study_kcap)
    mech = mechanism_for(w)
    m = rk.mech_load(mech)
    n = 1024
    U_all = initial_state(w, n_cells=1 << 16)
    U0 = torch.tensor(U_all[np.linspace(0, U_all.shape[0] - 1, n).astype(np.int64)], device=dev)
    ns = mech.n_species
    T_END = 1e-5
    rtol, atol = 1e-4, 1e-8
    st = torch.zeros(n, 4, dtype=torch.int32, device=dev)

    def run(method, M, h_cfl, rt, at, jv_mode=0):
        Y = U0.clone()
        hc = torch.zeros(n, dtype=torch.float64, device=dev)
        tot = np.zeros(4, dtype=np.int64)
        ws = torch.empty(rk.rok4e_workspace_size(m, n, M), dtype=torch.uint8, device=dev)
        o = rk.Opts(jv_mode=jv_mode)
        n_int = int(round(T_END / h_cfl))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(n_int):
            if method == "rkdp":
                rk.rkdp_integrate(m, Y, h_cfl, rt, at, h_cell=hc, opts=o, stats=st, workspace=ws)
            else:
                rk.rok4e_integrate(m, Y, h_cfl, rt, at, M, h_cell=hc, opts=o, stats=st, workspace=ws)
            if n_int <= 100:
                tot += st.sum(dim=0).cpu().numpy()
        e1.record()
        torch.cuda.synchronize()
        return Y, e0.elapsed_time(e1) * 1e-3, tot, n_int

    ref, t_ref, _, _ = run("rok4e", 8, 1e-6, 1e-10, 1e-14)
    ref_dp, _, _, _ = run("rkdp", 1, 1e-6, 1e-10, 1e-14)
    Tref = ref[:, ns]
    ref_check = float(((ref_dp[:, ns] - Tref).abs() / Tref).max())
    cases = [("rok4e", 4, 0), ("rok4e", 6, 0), ("rok4e", 8, 0), ("rok4e", 4, 1), ("rkdp", 1, 0)]
    for h_cfl in (1e-9, 1e-8, 1e-7, 1e-6, 1e-5):
        for method, M, jv in cases:
            Y, t, tot, n_int = run(method, M, h_cfl, rtol, atol, jv)
            rel = ((Y[:, ns] - Tref).abs() / Tref).cpu().numpy()
            name = "RKDP" if method == "rkdp" else f"ROK4E M={M}" + (" FD J v" if jv else "")
            line = {"study": "efficiency", "k_cap": w.k_cap, "method": name, "h_cfl_s": h_cfl, "intervals": n_int,
                    "cells": n, "horizon_s": T_END, "rtol": rtol, "atol": atol,
                    "gpu_s": t, "gpu_us_per_cell": t / n * 1e6,
                    "T_rel_err_max": float(rel.max()), "T_rel_err_mean": float(rel.mean()),
                    "reference": "ROK4E M=8 rtol 1e-10 atol 1e-14",
                    "reference_vs_rkdp_T_rel": ref_check}
            if n_int <= 100:
                line.update({"attempts_per_cell": float((tot[0] + tot[1]) / n), "rhs_per_cell": float(tot[2] / n),
                             "failed": int(tot[3] != 0)})
            print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_1712_00953_gb300 as rk

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl", device_id=dev)
    w, mech, U0 = build_inputs(rank)
    npts, N = U0.shape
    dx = LENGTH / npts
    M = w.krylov_dim
    m = rk.mech_load(mech)
    stream = torch.cuda.current_stream()
    U = torch.tensor(U0, device=dev)
    hc = torch.zeros(npts, dtype=torch.float64, device=dev)
    ws = torch.empty(rk.simpler_split_step_workspace_size(m, npts, M), dtype=torch.uint8, device=dev)
    stats_all = torch.zeros(max(args.steps, 1), npts, 4, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in kev:  # materialise the events so their handles can be passed down
        a.record(stream)
        b.record(stream)

    def step(stats=None, events=None):
        rk.simpler_split_step(m, U, w.dt, D_DIFF, dx, w.rtol, w.atol, M, h_cell=hc, stats=stats,
                              opts=rk.Opts(events=events, lanes_per_cell=args.lanes, cells_per_block=args.cells_per_block, precision=PREC[args.precision], queue_order=args.queue_order, blocks_per_sm=args.blocks_per_sm), workspace=ws,
                              stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    U_start, hc_start = U.clone(), hc.clone()  # every pass below replays the same steps

    def restore():
        U.copy_(U_start)
        hc.copy_(hc_start)

    # ---- the split step captured once in a CUDA graph, replayed every step
    stats_step = torch.zeros(npts, 4, dtype=torch.int32, device=dev)
    graph = torch.cuda.CUDAGraph()
    cap_stream = torch.cuda.Stream(device=dev)
    cap_stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap_stream):
        with torch.cuda.graph(graph, stream=cap_stream, capture_error_mode="relaxed"):
            rk.simpler_split_step(m, U, w.dt, D_DIFF, dx, w.rtol, w.atol, M, h_cell=hc, stats=stats_step,
                                  opts=rk.Opts(lanes_per_cell=args.lanes, cells_per_block=args.cells_per_block, precision=PREC[args.precision], queue_order=args.queue_order, blocks_per_sm=args.blocks_per_sm), workspace=ws, stream=cap_stream)
    torch.cuda.current_stream().wait_stream(cap_stream)
    torch.cuda.synchronize()
    restore()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))  # evict the previous step's data from L2 (outside the timed events)
            ev[k][0].record(stream)
            graph.replay()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    U_graph = U.clone()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = max_over_ranks(sum(step_ms) * 1e-3, dist, dev)
    value = world * npts * args.steps / t_total

    # ---- roofline pass: the same steps launched eagerly, the integration
    # kernel bracketed by events on its own launch stream, per-step statistics
    restore()
    for k in range(args.steps):
        flush.fill_(float(k))
        step(stats_all[k], kev[k])
    torch.cuda.synchronize()
    kern_ms = [a.elapsed_time(b) for a, b in kev]
    graph_matches_eager = bool(torch.equal(U, U_graph))

    # ---- critical path: the reaction sub-step of the first timed step for all
    # cells, then for its most expensive cell alone (one warp on an otherwise
    # idle GPU): a launch cannot end before its hottest cell's serial
    # instruction stream has run
    restore()
    Tn = rk.diffusion_1d(U, D_DIFF, dx)
    cp_opts = rk.Opts(lanes_per_cell=args.lanes, cells_per_block=args.cells_per_block,
                      precision=PREC[args.precision], queue_order=args.queue_order,
                      blocks_per_sm=args.blocks_per_sm)
    cp_st = torch.zeros(npts, 4, dtype=torch.int32, device=dev)
    cp_ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    cp_t = []
    for cells in (None, "hottest"):
        if cells is None:
            Yc, hcc, srcc, stc = U.clone(), hc_start.clone(), Tn, cp_st
        else:
            c = int(torch.argmax(cp_st[:, 0] + cp_st[:, 1]).item())
            hot_attempts = int((cp_st[c, 0] + cp_st[c, 1]).item())
            Yc, hcc, srcc = U[c:c + 1].clone(), hc_start[c:c + 1].clone(), Tn[c:c + 1].contiguous()
            stc = torch.zeros(1, 4, dtype=torch.int32, device=dev)
        ts = []
        for _ in range(3):
            Y2, h2 = Yc.clone(), hcc.clone()
            flush.fill_(0.0)
            cp_ev[0].record(stream)
            rk.rok4e_integrate(m, Y2, w.dt, w.rtol, w.atol, M, src=srcc, h_cell=h2, opts=cp_opts, stats=stc,
                               stream=stream)
            cp_ev[1].record(stream)
            torch.cuda.synchronize()
            ts.append(cp_ev[0].elapsed_time(cp_ev[1]))
        cp_t.append(min(ts))
    critical_path = {"all_cells_ms": cp_t[0], "hottest_cell_alone_ms": cp_t[1],
                     "hottest_cell_attempts": hot_attempts, "ratio": cp_t[0] / cp_t[1],
                     "what": "reaction sub-step of the first timed split step: whole grid vs its most expensive "
                             "cell integrated alone"}

    # ---- end to end through the public API with host buffers: the same steps
    # from the same state, with the state copied in from pinned host memory and
    # the result copied back every step
    restore()
    pinned = U_start.cpu().pin_memory()
    e2e_steps = args.steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(e2e_steps):
        U.copy_(pinned, non_blocking=True)
        step()
        pinned.copy_(U, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_t = e0.elapsed_time(e1) * 1e-3
    e2e_value = world * npts * e2e_steps / e2e_t
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return 0

    # ---- roofline of the dominant kernel (FP64 ALU)
    fma64 = rk.probe_throughput(0)
    exp64 = rk.probe_throughput(2)
    exp_fma = fma64 / exp64
    model = flop_model(mech, M)
    st = stats_all.cpu().numpy()
    flops = algorithmic_flops(model, st, M)
    kern_total = sum(kern_ms) * 1e-3
    achieved = flops / kern_total / 1e12
    peak_nominal = 1.25  # TFLOP/s FP64 (GB300 nominal)
    peak_meas = 2.0 * fma64 / 1e12
    bad = int((st[:, :, 3] != 0).sum())

    # ---- CPU baseline: the oracle on a bounded sample of the initial field
    cells = stratified_cells(npts, args.cpu_cells)
    cpu_v, cpu_t, U_react_ref = cpu_oracle_sample(w, mech, U0, cells)
    # accuracy on the same sample: the GPU's reaction sub-step of the first
    # split step (constant source T(U_n)) against the oracle's, both running
    # their own adaptive step sequences from h = dt
    Ug = torch.tensor(U0, device=dev)
    Yr = Ug.clone()
    rk.rok4e_integrate(m, Yr, w.dt, w.rtol, w.atol, M, src=rk.diffusion_1d(Ug, D_DIFF, dx),
                       opts=rk.Opts(precision=PREC[args.precision]))
    Yr = Yr.cpu().numpy()[cells]
    Rr = U_react_ref[cells]
    ns = mech.n_species
    dY = np.abs(Yr[:, :ns] - Rr[:, :ns])
    dT = np.abs(Yr[:, ns] - Rr[:, ns])
    accuracy = {"vs": "FP64 oracle, reaction sub-step of the first split step, free-running step sequences",
                "cells": len(cells), "max_abs_dY": float(dY.max()),
                "max_rel_dY_where_Y_gt_1e-8": float((dY / np.maximum(np.abs(Rr[:, :ns]), 1e-8)).max()),
                "max_abs_dT_K": float(dT.max()),
                "within_1e-8_plus_1e-6Y_and_1e-6K": bool(np.all(dY <= 1e-8 + 1e-6 * np.abs(Rr[:, :ns]))
                                                         and np.all(dT <= 1e-6))}

    cpu_all_v, cpu_all_procs, cpu_all_t = cpu_oracle_sample_all_cores(w, mech, U0, cells)

    clocks = clk.summary()
    line = {
        "metric": "cell-steps/s", "value": value, "unit": "cell-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f64+f32 (mixed)", "data": "synthetic",
        "config": {"workload": "flame1d 1-D reaction-diffusion, 2048 points, 30 species / 150 reactions "
                               "(4 third-body, 2 Troe), Simpler split steps of 1e-7 s, ROK4E M=4, rtol 1e-6, "
                               "atol 1e-10", "precision": args.precision, "points": npts,
                   "l2": "flushed (256 MB write) between steps", "parallelism": f"replicas x{world}",
                   "lanes_per_cell": args.lanes or 32, "cells_per_block": args.cells_per_block,
                   "queue_order": args.queue_order, "blocks_per_sm": args.blocks_per_sm},
        # traffic: dram__bytes_read.sum + dram__bytes_write.sum of one fp64
        # integration launch of this workload from one ncu --set full capture
        # of the current kernel (bytes per launch), null while no capture of
        # the current kernel exists; traffic_last_capture keeps the figure of
        # the last captured build, labelled as such
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_nominal, "unit": "TFLOP/s",
                     "frac": achieved / peak_nominal,
                     "traffic": None,
                     "traffic_last_capture": {"bytes_per_launch": 1531904, "build": "before the cell slots "
                                              "dropped the double-float arrays outside precision level 3 "
                                              "(shared-memory offsets only)"} if args.precision == "fp64" else None,
                     "traffic_unit": "bytes per launch (ncu capture)",
                     "algorithmic_bytes_per_launch": int(npts * N * 8 * 3 + npts * (16 + 16)),
                     "kernel": "rok4e_integrate_kernel<32>", "kernel_ms_per_step": 1e3 * kern_total / args.steps,
                     "peak_probe_fp64": peak_meas, "frac_of_probe": achieved / peak_meas,
                     "exp_flops_counted": EXP_FLOPS, "cuda_exp_cost_fma_measured": exp_fma,
                     "algorithmic_tflop_per_step": flops / args.steps / 1e12},
        "accuracy": accuracy,
        "critical_path": critical_path,
        "cpu_baseline": {"value": cpu_v, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.cpu_cells} cells spread over the grid (golden-ratio sequence), one "
                                   f"split step of the initial field ({cpu_t:.1f} s)"},
        "cpu_baseline_all_cores": {"value": cpu_all_v, "unit": "cell-steps/s", "cores": cpu_all_procs,
                                   "kind": "oracle",
                                   "sample": f"the same {len(cells)} cells' reaction sub-steps, one process per core "
                                             f"({cpu_all_t:.1f} s)"},
        "e2e": {"value": e2e_value, "unit": "cell-steps/s", "h2d_bytes_per_step": int(U.numel() * 8),
                "d2h_bytes_per_step": int(U.numel() * 8), "steps": e2e_steps},
        # per split step: diffusion, the three queue-ordering kernels (longest-first
        # orders), the integration, three SSP-RK3 stages
        "gpu_launches": (5 + (3 if args.queue_order in (0, 2, 3) else 0)) * args.steps,
        "cuda_graph": {"timed_region": "one captured split step replayed per step",
                       "matches_eager_bitwise": graph_matches_eager},
        "clocks": clocks,
        "cells_failed": bad,
        "substeps_per_cell_step": float(st[:, :, 0].mean()),
        "max_substeps_per_cell_step": int(st[:, :, 0].max()),
        "attempts_per_cell_step": float((st[:, :, 0] + st[:, :, 1]).mean()),
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-cells", type=int, default=48)
    ap.add_argument("--plain-steps", type=int, default=0,
                    help="run this many untimed split steps and exit (profiling case)")
    ap.add_argument("--lanes", type=int, default=0, help="lanes per cell (0: library default)")
    ap.add_argument("--cells-per-block", type=int, default=8, help="cells per block (0: library default)")
    ap.add_argument("--precision", default="fp64", choices=list(PREC))
    ap.add_argument("--queue-order", type=int, default=3, help="0 auto, 1 interleaved, 2 longest first, 3 static balanced bins")
    ap.add_argument("--unit-costs", action="store_true",
                    help="small RHS / J v / integration launches (for ncu instruction counts) and the probes")
    ap.add_argument("--skip-probes", action="store_true")
    ap.add_argument("--study-kcap", type=float, default=0.0,
                    help="efficiency study on a variant of the batched mechanism with this cap on k C (1/s)")
    ap.add_argument("--study", default="", choices=["", "efficiency"],
                    help="efficiency: the ROK4E M / J v mode / explicit RK comparison over h_CFL")
    ap.add_argument("--workload", default="flame1d", choices=["flame1d", "batched"],
                    help="flame1d: the benchmark line; batched: the 2^20-cell throughput measurement")
    ap.add_argument("--blocks-per-sm", type=int, default=0, help="resident blocks per SM (0: all that fit)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.plain_steps > 0:
        return run_plain(args)
    if args.unit_costs:
        return run_unit_costs(args)
    if args.study == "efficiency":
        return run_study(args, local_rank)
    if args.workload == "batched":
        return run_batched(args, rank, world, local_rank)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
