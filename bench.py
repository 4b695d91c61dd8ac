"""Benchmark: the ROK4E reaction step over 2^20 independent cells, plus the
other four workloads as keyed blocks of the same JSON line.

Headline (``value``): the batched workload -- 2^20 constant-pressure cells cut
from a seeded 128^3 Gaussian random temperature field (mean 1400 K, std 300 K),
a 53-species / 325-reaction synthetic mechanism, one reaction step of
dt = 1e-6 s per cell (rtol 1e-6, atol 1e-10), FP64.  One bench step restores
the initial field and the per-cell step sizes carried from one earlier step
and integrates every cell over dt in one persistent launch; the restore and
the launch are captured once in a CUDA graph and replayed.  The Krylov
dimension (4..8) and the launch shape are chosen by the autotuner on a sample
of the cells.  Metric: cell-steps/s = cells x steps / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Keyed blocks under "configs" (N = 1 only): ``small`` (10 species / 24
reactions, 256 cells, one 1e-6 s step), ``flame1d`` (1-D reaction-diffusion,
2048 points, 30 / 150 with 4 third-body and 2 Troe reactions, Simpler split
steps of 1e-7 s), ``mixed`` (the flame1d workload at precision levels 1-3),
``adjoint`` (4096 cells, 100 / 500, 50 fixed steps of 1e-7 s, forward with
checkpoints and the adjoint of the final temperatures w.r.t. ln A).

Under torchrun (N > 1) every rank integrates its own 2^20 cells (a field
seeded per rank): weak scaling, no data-path collective; the time is the
slowest rank's.  ``--impl reference`` times the FP64 numpy oracle on the host
cores on a bounded sample of the headline workload (rank 0 only): the
compiled C oracle on every host core.  Every CPU baseline in the line is an
oracle as it stands (the C oracle at -O3 on all cores and on one, and the
numpy oracle on one core), on a stated sample of the same workload.
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

D_DIFF = 1.0e-4  # m^2/s
LENGTH = 1.0e-2  # m
P_ATM = 101325.0
L2_FLUSH_BYTES = 256 << 20
PREC = {"fp64": 0, "mixed": 1, "mixed-fp32jv": 2, "mixed-df": 3, "tensor": 4, "exp32": 5, "fp32jv": 6}
FP64_PEAK = 1.25  # TFLOP/s: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal)
GOLDEN = 0.6180339887498949

# dram__bytes_read.sum + dram__bytes_write.sum of one integration launch from
# an ncu capture of the current kernel (bytes per launch), keyed by workload;
# None while no capture of the current kernel exists.  The last captures are of
# the build before the Krylov-dimension loops were made compile-time (a change
# that moves no data): batched 280,948,224 B per 2^18-cell launch, i.e.
# 1,123,792,896 B scaled by cells to the 2^20-cell launch; flame1d 2,118,656 B
# for the 8th split step's launch, whose 0.5 MB state stays in L2.
TRAFFIC = {"batched": None, "flame1d": None}


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


# ------------------------------------------------------------- work model
def flop_model(mech, M):
    """Algorithmic FP64 operation counts (flops, FMA = 2) of the kernels' units.

    Returns dict(rhs, rhs_exp, jvp, arnoldi, attempt) per unit.  Transcendentals
    are counted separately (rhs_exp) and converted with EXP_FLOPS."""
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


def adjoint_flop_model(mech, M):
    """Algorithmic FP64 flops of the adjoint of one fixed ROK4E step of one
    cell (rk_rok4e_adjoint), FMA = 2, one exp or log = EXP_FLOPS, a division 1.

    Value passes of the right-hand side: per species 46 (thermo polynomials,
    C, the sums of the temperature equation, f), per net coefficient 2 (the
    gather), per reaction 16 plus 6 for a reversible one, two exponentials per
    reversible reaction and one per other, 2 per species and third-body
    reaction.  Their reverse: per species 34 plus 3 per reaction slot the
    species fills, per reaction 26.  A dual (value, tangent) pass costs 2.5x
    its value pass's arithmetic plus one multiply per exponential.  Per step:
    3 value and M dual forward passes (f at u_n and at the two stage
    arguments, and the M J q_j; every tape is kept for the reverse sweep), 3
    value and M dual reverse passes; the Krylov and stage algebra forward and
    reverse three times the forward step's (the integrator's Arnoldi and
    attempt counts)."""
    ns, nr = mech.n_species, mech.n_reactions
    kind = np.asarray(mech.kind)
    rev = np.asarray(mech.reversible).astype(bool)
    n_tb = int((kind > 0).sum())
    n_rev = int(rev.sum())
    slots = int(sum(sum(abs(int(n)) for s_, n in zip(mech.rxn_sp[j], mech.rxn_nu[j]) if s_ >= 0) for j in range(nr)))
    fm = flop_model(mech, M)
    nnz_term = fm["rhs"] - (ns * 40 + nr * 16 + n_tb * 2 * ns + 10)  # 2 per net coefficient (+ Troe)
    fwd_v = ns * 46 + nnz_term + nr * 16 + n_rev * 6 + n_tb * 2 * ns
    exps = nr + n_rev
    rev_v = ns * 34 + 3 * slots + nr * 26
    fwd_d = 2.5 * fwd_v + exps
    rev_d = 2.5 * rev_v
    krylov = 3 * (fm["arnoldi"] + fm["attempt"])
    return float(3 * (fwd_v + EXP_FLOPS * exps) + M * (fwd_d + EXP_FLOPS * exps) + 3 * rev_v + M * rev_d + krylov)


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


# ---------------------------------------------------------------- oracle legs
def golden_cells(n, count, offset=1):
    """count distinct cell indices spread over [0, n) (golden-ratio sequence)."""
    out, seen, i = [], set(), offset
    while len(out) < min(count, n):
        c = int(i * GOLDEN * n) % n
        if c not in seen:
            seen.add(c)
            out.append(c)
        i += 1
    return out


def _oracle_cell(task):
    """One cell through the oracle (worker process): ROK4E over dt from u0 with
    an optional constant source, first step h0 (None: dt)."""
    from oracle import rok4e
    from oracle.kinetics import Kinetics

    mech, u0, src, dt, rtol, atol, M, h0 = task
    f, jv_at = rok4e.reactor(Kinetics(mech), P_ATM, src)
    return rok4e.integrate(f, jv_at, u0, dt, rtol, atol, M, h0=h0)[0]


def oracle_time(tasks, procs):
    """Wall time of the oracle on the tasks, in `procs` spawned processes
    (no CUDA state is inherited); procs = 1 runs in this process."""
    if procs <= 1:
        t0 = time.perf_counter()
        for t in tasks:
            _oracle_cell(t)
        return time.perf_counter() - t0
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_cell, tasks[:procs])  # start-up (imports) outside the timing
        t0 = time.perf_counter()
        pool.map(_oracle_cell, tasks, chunksize=1)
        return time.perf_counter() - t0


def c_oracle_rate(mech, U, src, h0, dt, rtol, atol, M, threads):
    """Cells per second of the C oracle (gcc -O3, OpenMP over cells) integrating
    the rows of U over dt on `threads` host threads (a short untimed run first)."""
    from oracle import c_oracle

    co = c_oracle.COracle(mech)
    k = min(len(U), max(1, threads))
    co.integrate(U[:k], dt, rtol, atol, M, src=None if src is None else src[:k],
                 h0=None if h0 is None else h0[:k], threads=threads)
    t0 = time.perf_counter()
    co.integrate(U, dt, rtol, atol, M, src=src, h0=h0, threads=threads)
    t = time.perf_counter() - t0
    return len(U) / t, t


def cpu_baselines(mech, U, src, h0, dt, rtol, atol, M, n_single, what):
    """cpu_baseline (the C oracle on every host core), plus the same oracle on
    one core and the numpy oracle on one core, on cells spread over the
    workload (golden-ratio sequence over the rows of U)."""
    n = U.shape[0]
    procs = max(1, os.cpu_count() or 1)

    def sample(count):
        c = golden_cells(n, count, offset=101)
        return U[c], None if src is None else src[c], None if h0 is None else h0[c]

    Um, sm, hm = sample(n_single * procs)
    vm, tm = c_oracle_rate(mech, Um, sm, hm, dt, rtol, atol, M, procs)
    U1, s1, h1 = sample(n_single)
    v1, t1 = c_oracle_rate(mech, U1, s1, h1, dt, rtol, atol, M, 1)
    Un, sn, hn = sample(4)
    tn = oracle_time([(mech, Un[i], None if sn is None else sn[i], dt, rtol, atol, M,
                       None if hn is None else float(hn[i])) for i in range(len(Un))], 1)
    return {
        "cpu_baseline": {"value": vm, "unit": "cell-steps/s", "cores": procs, "kind": "oracle",
                         "sample": f"{len(Um)} {what}, the C oracle (gcc -O3, OpenMP over cells) on {procs} host "
                                   f"threads ({tm:.1f} s)"},
        "cpu_baseline_1core": {"value": v1, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
                               "sample": f"{len(U1)} of those cells, the C oracle on one thread ({t1:.1f} s)"},
        "cpu_baseline_numpy": {"value": len(Un) / tn, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
                               "sample": f"{len(Un)} of those cells, the numpy oracle on one core ({tn:.1f} s)"},
    }


def replay_accuracy(mech, U0, src, out, trace, cells, dt, rtol, atol, M, what):
    """The oracle replaying the GPU's recorded step sequences of `cells`:
    max |dY|, max relative dY, max |dT|, per-species maxima, and the bar
    |dY| <= 1e-8 + 1e-6 |Y|, |dT| <= 1e-6 K."""
    from oracle import rok4e as orok
    from oracle.kinetics import Kinetics

    replay = [[(abs(h), h > 0) for h in trace[i] if h != 0.0] for i in range(len(cells))]
    ref, _ = orok.integrate_cells(Kinetics(mech), U0, P_ATM, dt, rtol, atol, M,
                                  src=src, replay=replay)
    ns = mech.n_species
    dY = np.abs(out[:, :ns] - ref[:, :ns])
    dT = np.abs(out[:, ns] - ref[:, ns])
    return {"vs": f"FP64 oracle replaying the GPU's step sequences ({what})", "cells": len(cells),
            "max_abs_dY": float(dY.max()),
            "max_rel_dY_where_Y_gt_1e-8": float((dY / np.maximum(np.abs(ref[:, :ns]), 1e-8)).max()),
            "max_abs_dT_K": float(dT.max()),
            "per_species_max_abs_dY": [float(x) for x in dY.max(axis=0)],
            "within_1e-8_plus_1e-6Y_and_1e-6K": bool(np.all(dY <= 1e-8 + 1e-6 * np.abs(ref[:, :ns]))
                                                     and np.all(dT <= 1e-6))}


# ---------------------------------------------------------------- headline
def batched_field(w, rank, n_cells=None):
    """The batched workload's initial state for one rank (rank 0: the workload's
    own seed); ``n_cells`` keeps a prefix."""
    from synth.fields import field_gaussian3d

    return np.ascontiguousarray(field_gaussian3d(w.n_species, w.field_seed + 97 * rank, n_cells=n_cells))


def run_headline(args, rank, world, dev, dist):
    """The 2^20-cell batched step (see the module docstring).  Returns the
    fields of the JSON line (complete on rank 0)."""
    import torch

    import paper_1712_00953_gb300 as rk
    from paper_1712_00953_gb300 import autotune
    from synth.fields import WORKLOADS, mechanism_for

    w = WORKLOADS["batched"]
    mech = mechanism_for(w)
    U_host = batched_field(w, rank)
    n, N = U_host.shape
    m = rk.mech_load(mech)
    U0 = torch.tensor(U_host, device=dev)
    stream = torch.cuda.current_stream()

    # ---- autotuner: Krylov dimension 4..8 under an accuracy constraint, and the launch shape
    tune = None
    if args.no_autotune:
        M, lanes, cpb = (args.krylov or w.krylov_dim), args.lanes, args.cells_per_block
    else:
        samp = torch.tensor(U_host[golden_cells(n, args.tune_cells)], device=dev)
        tune = autotune.tune_krylov_and_shape(m, samp, w.dt, w.rtol, w.atol, dims=(4, 5, 6, 8),
                                              precision=PREC[args.precision], cache_path=None)
        M, lanes, cpb = tune["M"], tune["lanes_per_cell"], tune["cells_per_block"]
        if args.krylov:
            M = args.krylov
    opts_kw = dict(lanes_per_cell=lanes, cells_per_block=cpb, precision=PREC[args.precision],
                   queue_order=args.queue_order, blocks_per_sm=args.blocks_per_sm)

    Y = torch.empty_like(U0)
    hc = torch.zeros(n, dtype=torch.float64, device=dev)
    st = torch.zeros(n, 4, dtype=torch.int32, device=dev)
    ws = torch.empty(rk.rok4e_workspace_size(m, n, M), dtype=torch.uint8, device=dev)
    # one earlier step gives every cell its carried step size (h_snap)
    Y.copy_(U0)
    rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, M, h_cell=hc, opts=rk.Opts(**opts_kw), stats=st, workspace=ws)
    torch.cuda.synchronize()
    h_snap = hc.clone()

    kev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for e in kev:  # materialise the events so their handles can be passed down
        e.record(stream)
    torch.cuda.synchronize()

    def step(s=None):
        Y.copy_(U0)
        hc.copy_(h_snap)
        rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, M, h_cell=hc, opts=rk.Opts(events=kev, **opts_kw),
                           stats=st, workspace=ws, stream=s)

    for _ in range(args.warmup - 1):
        step()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    cap_stream = torch.cuda.Stream(device=dev)
    cap_stream.wait_stream(stream)
    with torch.cuda.stream(cap_stream):
        with torch.cuda.graph(graph, stream=cap_stream, capture_error_mode="relaxed"):
            step(cap_stream)
    stream.wait_stream(cap_stream)
    torch.cuda.synchronize()
    graph.replay()  # the captured step once more, untimed (checks it runs)
    torch.cuda.synchronize()
    Y_warm = Y.clone()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    step_ms, kern_ms = [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        for k in range(args.steps):
            ev[k][0].record(stream)
            graph.replay()
            ev[k][1].record(stream)
            torch.cuda.synchronize()
            step_ms.append(ev[k][0].elapsed_time(ev[k][1]))
            try:
                kern_ms.append(kev[0].elapsed_time(kev[1]))
            except RuntimeError:
                kern_ms.append(None)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_total = max_over_ranks(sum(step_ms) * 1e-3, dist, dev)
    value = world * n * args.steps / t_total
    same_every_step = bool(torch.equal(Y, Y_warm))
    st_np = st.cpu().numpy()
    tot = reduce_stats(st_np, dist, dev)
    model = flop_model(mech, M)
    flops = algorithmic_flops(model, st_np, M)
    kern_valid = [x for x in kern_ms if x is not None]
    kernel_timing = "event-record nodes around the integration kernel inside the graph"
    if not kern_valid:
        kern_valid = step_ms
        kernel_timing = "graph replay (restore copies and ordering kernels included)"
    kern_s = statistics.mean(kern_valid) * 1e-3
    achieved = flops / kern_s / 1e12

    # ---- end to end through the public API with host buffers (pinned): every
    # step copies the initial state and carried steps in, integrates, and
    # copies the state back
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    pin_in = torch.from_numpy(U_host).pin_memory()
    pin_h = h_snap.cpu().pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(e2e_steps):
        Y.copy_(pin_in, non_blocking=True)
        hc.copy_(pin_h, non_blocking=True)
        rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, M, h_cell=hc, opts=rk.Opts(**opts_kw), stats=st,
                           workspace=ws)
        pin_out.copy_(Y, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_t = max_over_ranks(e0.elapsed_time(e1) * 1e-3, dist, dev)
    e2e_value = world * n * e2e_steps / e2e_t
    e2e_matches = bool(torch.equal(pin_out, Y_warm.cpu()))
    if rank != 0:
        return None

    # ---- accuracy: the 4 cells with the most attempts and 12 spread over the
    # field, integrated again alone with their step sequences recorded (a
    # cell's bits do not depend on the launch), replayed through the oracle
    att = st_np[:, 0] + st_np[:, 1]
    hot = [int(c) for c in np.argsort(-att, kind="stable")[:4]]
    cells = hot + [c for c in golden_cells(n, 16) if c not in hot][:12]
    Ys = U0[cells].clone()
    hs = h_snap[cells].clone()
    cap = int(att.max()) + 8
    tr = torch.zeros(len(cells), cap, dtype=torch.float64, device=dev)
    rk.rok4e_integrate(m, Ys, w.dt, w.rtol, w.atol, M, h_cell=hs, opts=rk.Opts(trace=tr, **opts_kw))
    torch.cuda.synchronize()
    alone_matches = bool(torch.equal(Ys, Y_warm[cells]))
    accuracy = replay_accuracy(mech, U_host[cells], None, Ys.cpu().numpy(), tr.cpu().numpy(), cells, w.dt,
                               w.rtol, w.atol, M, "4 cells with the most attempts and 12 spread over the field")
    accuracy["sampled_cells_alone_bitwise_equal_full_launch"] = alone_matches

    # ---- CPU baselines: the oracles on cells spread over the field, each over
    # dt from its carried step (unbiased for the mean cost per cell)
    base = cpu_baselines(mech, U_host, None, h_snap.cpu().numpy(), w.dt, w.rtol, w.atol, M, args.cpu_cells,
                         "cells spread over the field, each over dt from its carried step")

    clocks = clk.summary()
    return {
        "metric": "cell-steps/s", "value": value, "unit": "cell-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f64+f32 (mixed)",
        "data": "synthetic (seeded)",
        "config": {"workload": "batched: 2^20 constant-pressure cells per GPU from a 128^3 Gaussian random "
                               "temperature field (mean 1400 K, std 300 K), 53 species / 325 reactions, one "
                               "ROK4E reaction step of 1e-6 s per cell, rtol 1e-6, atol 1e-10",
                   "cells_per_gpu": n, "krylov_dim": M, "precision": args.precision,
                   "lanes_per_cell": lanes or 32, "cells_per_block": cpb, "queue_order": args.queue_order,
                   "step": "restore the initial field and the step sizes carried from one earlier step, "
                           "integrate every cell over dt (one CUDA graph replay)",
                   "l2": "inputs larger than L2 (the 453 MB state is rewritten by the restore each step)",
                   "parallelism": f"dp{world} (independent fields per rank)",
                   "autotune": tune},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK, "peak_kind": "nominal FP64 (MEASURED_PEAKS.json has no FP64 "
                                                                "entry; the bench's own FMA probe agrees)",
                     "traffic": TRAFFIC["batched"],
                     "traffic_note": "null: no ncu capture of the current kernel; the previous build's "
                                     "2^18-cell capture scaled to 2^20 cells read and wrote 1.124e9 B "
                                     "(profiles/rok4e_integrate_batched.md)",
                     "algorithmic_bytes_per_launch": int(n * (2 * N * 8 + 16 + 8 + 8 + 4)),
                     "kernel": "rok4e_integrate_kernel<32, 0>", "kernel_s_per_step": kern_s,
                     "kernel_timing": kernel_timing, "exp_flops_counted": EXP_FLOPS,
                     "algorithmic_tflop_per_step": flops / 1e12},
        "accuracy": accuracy,
        **base,
        "e2e": {"value": e2e_value, "unit": "cell-steps/s", "h2d_bytes_per_step": int(n * N * 8 + n * 8),
                "d2h_bytes_per_step": int(n * N * 8), "steps": e2e_steps,
                "result_matches_device_run_bitwise": e2e_matches},
        # per step: the three queue-ordering kernels and the integration kernel
        "gpu_launches": 4 * args.steps,
        "cuda_graph": {"timed_region": "one captured step (restore + ordering + integration) replayed per step",
                       "identical_result_every_step": same_every_step},
        "clocks": clocks,
        "cells_failed": tot["failed_cells"],
        "substeps_per_cell_step": tot["accepted"] / tot["cells"],
        "max_substeps_per_cell_step": tot["substeps_max"],
        "attempts_per_cell_step": tot["attempts"] / tot["cells"],
        "attempts_per_s": world * tot["attempts"] / tot["cells"] * n * args.steps / t_total,
    }


# ---------------------------------------------------------------- flame1d (c2, c4)
def run_flame(args, dev, precision, extras=True):
    """Simpler split steps of the 1-D flame (2048 points, 30 / 150), a CUDA
    graph of one split step replayed for the K timed steps after W warm-up
    steps from the initial tanh field.  The rate depends on how far the flame
    has evolved, so the steps' window is stated and attempts/s is given too."""
    import torch

    import paper_1712_00953_gb300 as rk
    from synth.fields import WORKLOADS, field_tanh_front, mechanism_for

    w = WORKLOADS["flame1d"]
    mech = mechanism_for(w)
    _, U_host = field_tanh_front(w.n_cells, w.n_species, w.field_seed)
    npts, N = U_host.shape
    dx = LENGTH / npts
    M = w.krylov_dim
    m = rk.mech_load(mech)
    stream = torch.cuda.current_stream()
    U = torch.tensor(U_host, device=dev)
    hc = torch.zeros(npts, dtype=torch.float64, device=dev)
    ws = torch.empty(rk.simpler_split_step_workspace_size(m, npts, M), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    opts_kw = dict(lanes_per_cell=args.lanes, cells_per_block=args.flame_cells_per_block, precision=precision,
                   queue_order=args.queue_order, blocks_per_sm=args.blocks_per_sm)
    K = args.steps
    stats_all = torch.zeros(K, npts, 4, dtype=torch.int32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for a, b in kev:
        a.record(stream)
        b.record(stream)

    def step(stats=None, events=None, s=None):
        rk.simpler_split_step(m, U, w.dt, D_DIFF, dx, w.rtol, w.atol, M, h_cell=hc, stats=stats,
                              opts=rk.Opts(events=events, **opts_kw), workspace=ws, stream=s)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    U_start, hc_start = U.clone(), hc.clone()

    def restore():
        U.copy_(U_start)
        hc.copy_(hc_start)

    stats_step = torch.zeros(npts, 4, dtype=torch.int32, device=dev)
    graph = torch.cuda.CUDAGraph()
    cap_stream = torch.cuda.Stream(device=dev)
    cap_stream.wait_stream(stream)
    with torch.cuda.stream(cap_stream):
        with torch.cuda.graph(graph, stream=cap_stream, capture_error_mode="relaxed"):
            step(stats_step, None, cap_stream)
    stream.wait_stream(cap_stream)
    torch.cuda.synchronize()
    restore()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        for k in range(K):
            flush.fill_(float(k))  # evict the previous step's data from L2 (outside the timed events)
            ev[k][0].record(stream)
            graph.replay()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    U_graph = U.clone()
    t_total = sum(a.elapsed_time(b) for a, b in ev) * 1e-3
    value = npts * K / t_total

    # the same steps launched eagerly, the integration kernel bracketed by
    # events on its own stream, with per-step statistics
    restore()
    for k in range(K):
        flush.fill_(float(k))
        step(stats_all[k], kev[k])
    torch.cuda.synchronize()
    kern_total = sum(a.elapsed_time(b) for a, b in kev) * 1e-3
    graph_matches_eager = bool(torch.equal(U, U_graph))
    st = stats_all.cpu().numpy()
    model = flop_model(mech, M)
    flops = algorithmic_flops(model, st, M)
    achieved = flops / kern_total / 1e12
    attempts = float((st[:, :, 0] + st[:, :, 1]).sum())
    out = {"workload": "flame1d: 1-D reaction-diffusion, 2048 points on 1 cm, 30 species / 150 reactions "
                       "(4 third-body, 2 Troe), Simpler split steps of 1e-7 s, ROK4E M=4, rtol 1e-6, atol 1e-10",
           "precision": {v: k for k, v in PREC.items()}[precision],
           "value": value, "unit": "cell-steps/s", "steps": K, "warmup": args.warmup,
           "steps_window": f"split steps {args.warmup + 1}..{args.warmup + K} from the initial tanh field",
           "ms_per_step": 1e3 * t_total / K, "attempts_per_s": attempts / t_total,
           "attempts_per_cell_step": attempts / (K * npts),
           "substeps_per_cell_step": float(st[:, :, 0].mean()),
           "max_substeps_per_cell_step": int(st[:, :, 0].max()),
           "cells_failed": int((st[:, :, 3] != 0).sum()),
           "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK, "unit": "TFLOP/s",
                        "frac": achieved / FP64_PEAK, "traffic": TRAFFIC["flame1d"] if precision == 0 else None,
                        "algorithmic_bytes_per_launch": int(npts * N * 8 * 3 + npts * (16 + 16)),
                        "kernel": {0: "rok4e_integrate_kernel<32, 0, 0>", 3: "rok4e_integrate_kernel<32, 0, 0>",
                                   4: "rok4e_integrate_kernel<32, 0, 1>", 5: "rok4e_integrate_kernel<32, 0, 0>",
                                   6: "rok4e_integrate_kernel<32, 0, 0>"}.get(precision,
                                                                              "rok4e_integrate_kernel<32, 1, 0>"),
                        "kernel_ms_per_step": 1e3 * kern_total / K},
           "cuda_graph": {"timed_region": "one captured split step replayed per step",
                          "matches_eager_bitwise": graph_matches_eager},
           "gpu_launches": (5 + (3 if args.queue_order in (0, 2, 3) else 0)) * K,
           "clocks": clk.summary(),
           "l2": "flushed (256 MB write) between steps"}

    # accuracy: the reaction sub-step of the first split step from the initial
    # field (source T(U_n) from the oracle's transport, the same array on both
    # sides) on 8 points with the most attempts and 16 spread over the grid
    from oracle import splitting as osp

    src = osp.diffusion_op(U_host, D_DIFF, dx)
    Yr = torch.tensor(U_host, device=dev)
    st1 = torch.zeros(npts, 4, dtype=torch.int32, device=dev)
    tr = torch.zeros(npts, 512, dtype=torch.float64, device=dev)
    rk.rok4e_integrate(m, Yr, w.dt, w.rtol, w.atol, M, src=torch.tensor(src, device=dev), stats=st1,
                       opts=rk.Opts(trace=tr, precision=precision))
    torch.cuda.synchronize()
    s1 = st1.cpu().numpy()
    att = s1[:, 0] + s1[:, 1]
    hot = [int(c) for c in np.argsort(-att, kind="stable")[:8]]
    cells = hot + [c for c in golden_cells(npts, 24) if c not in hot][:16]
    out["accuracy"] = replay_accuracy(mech, U_host[cells], src[cells], Yr.cpu().numpy()[cells],
                                      tr.cpu().numpy()[cells], cells, w.dt, w.rtol, w.atol, M,
                                      "reaction sub-step of the first split step, 8 points with the most attempts "
                                      "and 16 spread over the grid")
    if not extras:
        return out

    # critical path: the reaction sub-step of the first timed step for all
    # points, then for its most expensive point alone
    restore()
    Tn = rk.diffusion_1d(U, D_DIFF, dx)
    cp_opts = rk.Opts(**opts_kw)
    cp_st = torch.zeros(npts, 4, dtype=torch.int32, device=dev)
    cp_ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    cp_t = []
    hot_attempts = 0
    for which in ("all", "hottest"):
        if which == "all":
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
    out["critical_path"] = {"all_cells_ms": cp_t[0], "hottest_cell_alone_ms": cp_t[1],
                            "hottest_cell_attempts": hot_attempts, "ratio": cp_t[0] / cp_t[1],
                            "what": "reaction sub-step of the first timed split step: whole grid vs its most "
                                    "expensive point integrated alone"}

    # end to end through the public API with host buffers
    restore()
    pinned = U_start.cpu().pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(K):
        U.copy_(pinned, non_blocking=True)
        step()
        pinned.copy_(U, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    out["e2e"] = {"value": npts * K / (e0.elapsed_time(e1) * 1e-3), "unit": "cell-steps/s",
                  "h2d_bytes_per_step": int(U.numel() * 8), "d2h_bytes_per_step": int(U.numel() * 8), "steps": K}

    # CPU baselines: the oracles' reaction sub-step of the first split step
    # (source T(U_n), from h = dt) on points spread over the grid
    out.update(cpu_baselines(mech, U_host, src, None, w.dt, w.rtol, w.atol, M, args.cpu_cells,
                             "points spread over the grid, reaction sub-step of the first split step"))
    return out


# ---------------------------------------------------------------- batched levels (c4 on c3)
def run_batched_levels(args, dev, M, lanes, cpb):
    """Every precision level on the same 2^18 cells of the batched field
    (golden-ratio subset), one restore + integration per timed step after one
    warm-up step, each cell over dt from the step size carried from that
    warm-up; accuracy: 8 cells (the 4 with the most attempts and 4 spread)
    replayed through the FP64 oracle."""
    import torch

    import paper_1712_00953_gb300 as rk
    from synth.fields import WORKLOADS, mechanism_for

    w = WORKLOADS["batched"]
    mech = mechanism_for(w)
    U_all = batched_field(w, 0)
    U_host = np.ascontiguousarray(U_all[sorted(golden_cells(U_all.shape[0], 1 << 18))])
    del U_all
    n = U_host.shape[0]
    m = rk.mech_load(mech)
    stream = torch.cuda.current_stream()
    U0 = torch.tensor(U_host, device=dev)
    ws = torch.empty(rk.rok4e_workspace_size(m, n, M), dtype=torch.uint8, device=dev)
    out = {"cells": n, "krylov_dim": M, "steps": args.level_steps}
    for name in ("fp64", "mixed", "mixed-fp32jv", "mixed-df", "tensor", "exp32", "fp32jv"):
        prec = PREC[name]
        kw = dict(lanes_per_cell=lanes, cells_per_block=cpb, precision=prec, queue_order=args.queue_order)
        if name == "tensor":  # one cell per warp; the nu^T tiles take shared memory: as many cells as fit
            kw.update(lanes_per_cell=32, cells_per_block=0)
        Y = U0.clone()
        hc = torch.zeros(n, dtype=torch.float64, device=dev)
        st = torch.zeros(n, 4, dtype=torch.int32, device=dev)
        rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, M, h_cell=hc, opts=rk.Opts(**kw), stats=st, workspace=ws)
        torch.cuda.synchronize()
        h_snap = hc.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t = 0.0
        for _ in range(args.level_steps):
            Y.copy_(U0)
            hc.copy_(h_snap)
            e0.record(stream)
            rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, M, h_cell=hc, opts=rk.Opts(**kw), stats=st,
                               workspace=ws)
            e1.record(stream)
            torch.cuda.synchronize()
            t += e0.elapsed_time(e1) * 1e-3
        s_np = st.cpu().numpy()
        att = s_np[:, 0] + s_np[:, 1]
        hot = [int(c) for c in np.argsort(-att, kind="stable")[:4]]
        cells = hot + [c for c in golden_cells(n, 8, offset=3) if c not in hot][:4]
        tr = torch.zeros(len(cells), int(att.max()) + 8, dtype=torch.float64, device=dev)
        Ys = U0[cells].clone()
        rk.rok4e_integrate(m, Ys, w.dt, w.rtol, w.atol, M, h_cell=h_snap[cells].clone(),
                           opts=rk.Opts(trace=tr, **kw))
        torch.cuda.synchronize()
        acc = replay_accuracy(mech, U_host[cells], None, Ys.cpu().numpy(), tr.cpu().numpy(), cells, w.dt, w.rtol,
                              w.atol, M, "4 cells with the most attempts and 4 spread")
        out[name] = {"value": n * args.level_steps / t, "unit": "cell-steps/s",
                     "attempts_per_cell_step": float(att.mean()), "cells_failed": int((s_np[:, 3] != 0).sum()),
                     "accuracy": acc}
    for name in ("mixed", "mixed-fp32jv", "mixed-df", "tensor", "exp32", "fp32jv"):
        out[name]["vs_fp64"] = out[name]["value"] / out["fp64"]["value"]
    return out


# ---------------------------------------------------------------- small (c1)
def run_small(args, dev):
    """256 cells of the 10 / 24 mechanism, one ROK4E step of 1e-6 s from the
    initial field (h0 = dt), restore + integrate captured in a CUDA graph and
    replayed; all 256 cells replayed through the oracle."""
    import torch

    import paper_1712_00953_gb300 as rk
    from synth.fields import WORKLOADS, initial_state, mechanism_for

    w = WORKLOADS["small"]
    mech = mechanism_for(w)
    U_host = initial_state(w)
    n = U_host.shape[0]
    m = rk.mech_load(mech)
    stream = torch.cuda.current_stream()
    U0 = torch.tensor(U_host, device=dev)
    Y = torch.empty_like(U0)
    st = torch.zeros(n, 4, dtype=torch.int32, device=dev)
    ws = torch.empty(rk.rok4e_workspace_size(m, n, w.krylov_dim), dtype=torch.uint8, device=dev)

    def step(s=None):
        Y.copy_(U0)
        rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, w.krylov_dim, stats=st, workspace=ws, stream=s)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    cap_stream = torch.cuda.Stream(device=dev)
    cap_stream.wait_stream(stream)
    with torch.cuda.stream(cap_stream):
        with torch.cuda.graph(graph, stream=cap_stream, capture_error_mode="relaxed"):
            step(cap_stream)
    stream.wait_stream(cap_stream)
    torch.cuda.synchronize()
    reps = max(20, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) * 1e-3
    s = st.cpu().numpy()
    tr = torch.zeros(n, 1024, dtype=torch.float64, device=dev)
    Yt = U0.clone()
    rk.rok4e_integrate(m, Yt, w.dt, w.rtol, w.atol, w.krylov_dim, opts=rk.Opts(trace=tr))
    torch.cuda.synchronize()
    acc = replay_accuracy(mech, U_host, None, Yt.cpu().numpy(), tr.cpu().numpy(), list(range(n)), w.dt, w.rtol,
                          w.atol, w.krylov_dim, "all 256 cells")
    base = cpu_baselines(mech, U_host, None, None, w.dt, w.rtol, w.atol, w.krylov_dim, 64, "of the 256 cells")
    return {"workload": "small: 256 cells, 10 species / 24 reactions, T ~ U(1000, 1500) K, one ROK4E step of "
                        "1e-6 s, M=4, rtol 1e-6, atol 1e-10",
            "value": n * reps / t, "unit": "cell-steps/s", "steps": reps, "ms_per_step": 1e3 * t / reps,
            "attempts_per_cell_step": float((s[:, 0] + s[:, 1]).mean()), "cells_failed": int((s[:, 3] != 0).sum()),
            "cuda_graph": "restore + integration captured once, replayed per step",
            "gpu_launches": reps, "accuracy": acc, **base}


# ---------------------------------------------------------------- adjoint (c5)
def run_adjoint(args, dev):
    """4096 cells, 100 / 500, 50 fixed ROK4E steps of 1e-7 s: the forward
    with one checkpoint per step, then the adjoint of sum_c T_c(final) w.r.t.
    all ln A_j; the gradient along a random direction against GPU central
    differences (h = 1e-6) over all cells and the oracle's complex-step
    directional derivative on the coldest cell."""
    import torch

    import paper_1712_00953_gb300 as rk
    from synth.fields import WORKLOADS, initial_state, mechanism_for

    w = WORKLOADS["adjoint"]
    mech = mechanism_for(w)
    U_host = initial_state(w)
    n, N = U_host.shape
    h, nsteps, M = w.dt, w.n_steps, w.krylov_dim
    m = rk.mech_load(mech)
    stream = torch.cuda.current_stream()
    U0 = torch.tensor(U_host, device=dev)
    Y = torch.empty_like(U0)
    ck = torch.empty(nsteps + 1, n, N, dtype=torch.float64, device=dev)
    ubar = torch.zeros_like(U0)
    ubar[:, -1] = 1.0
    wsf = torch.empty(rk.rok4e_workspace_size(m, n, M), dtype=torch.uint8, device=dev)
    wsb = torch.empty(rk.rok4e_adjoint_workspace_size(m, n, M), dtype=torch.uint8, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tf, tb = [], []
    for rep in range(max(2, args.adjoint_reps)):
        Y.copy_(U0)
        torch.cuda.synchronize()
        ev[0].record(stream)
        rk.rok4e_fixed_steps(m, Y, h, nsteps, M, checkpoints=ck, workspace=wsf)
        ev[1].record(stream)
        grad, _ = rk.rok4e_adjoint(m, ck, ubar, h, nsteps, M, workspace=wsb)
        ev[2].record(stream)
        torch.cuda.synchronize()
        if rep > 0:  # the first repetition warms up
            tf.append(ev[0].elapsed_time(ev[1]) * 1e-3)
            tb.append(ev[1].elapsed_time(ev[2]) * 1e-3)
    t_f, t_b = statistics.mean(tf), statistics.mean(tb)
    # the adjoint alone at each lane count (one cell per 8, 16 or 32 lanes)
    sweep = {}
    for G in (4, 8, 16, 32):
        ts = []
        for rep in range(2):
            ev[1].record(stream)
            g_G, _ = rk.rok4e_adjoint(m, ck, ubar, h, nsteps, M, workspace=wsb, lanes_per_cell=G)
            ev[2].record(stream)
            torch.cuda.synchronize()
            if rep > 0:
                ts.append(ev[1].elapsed_time(ev[2]) * 1e-3)
        sweep[str(G)] = {"adjoint_s": min(ts),
                         "max_rel_diff_vs_auto": float((g_G - grad).abs().max() / grad.abs().max())}
    d = np.random.default_rng(7).normal(size=mech.n_reactions)
    d /= np.linalg.norm(d)
    # central differences along d on the GPU, per cell, at h = 1e-6 and 1e-7
    # in ln A: the fixed-step map is strongly nonlinear in some cells (hot
    # cells near instability), so the check uses the cells where the two
    # agree to 1e-3 (the converged finite differences)
    fd = {}
    for hd in (1e-6, 1e-7):
        vals = []
        for sgn in (1.0, -1.0):
            mk = mech.copy()
            mk.arrh[:, 0] = mk.arrh[:, 0] * np.exp(sgn * hd * d)
            mm = rk.mech_load(mk)
            Yd = U0.clone()
            rk.rok4e_fixed_steps(mm, Yd, h, nsteps, M, workspace=wsf)
            vals.append(Yd[:, -1].cpu().numpy())
        fd[hd] = (vals[0] - vals[1]) / (2 * hd)
    conv = np.abs(fd[1e-6] - fd[1e-7]) <= 1e-3 * np.abs(fd[1e-7])
    ubs = torch.zeros_like(U0)
    ubs[torch.tensor(np.nonzero(conv)[0], device=dev), -1] = 1.0
    gs, _ = rk.rok4e_adjoint(m, ck, ubs, h, nsteps, M, workspace=wsb)
    got_s = float(gs.cpu().numpy() @ d)
    fd_s = float(fd[1e-6][conv].sum())
    # the oracle's complex-step derivative (exact for the discrete map) on the
    # coldest cell and the median-temperature cell, each alone
    from oracle import adjoint as oad
    from oracle.kinetics import Kinetics

    kin = Kinetics(mech)
    lnA = kin.lnA_input.astype(complex) + 1j * oad.CS_EPS * d
    order = np.argsort(U_host[:, -1])
    cs_cells = []
    for c in (int(order[0]), int(order[len(order) // 2])):
        ub1 = torch.zeros_like(U0)
        ub1[c, -1] = 1.0
        g1, _ = rk.rok4e_adjoint(m, ck, ub1, h, nsteps, M, workspace=wsb)
        t0 = time.perf_counter()
        uf = oad.final_state(kin, U_host[c].astype(complex), P_ATM, h, nsteps, M, lnA)
        ref1 = float(np.imag(uf[-1])) / oad.CS_EPS
        got1 = float(g1.cpu().numpy() @ d)
        cs_cells.append({"cell": c, "T0_K": float(U_host[c, -1]), "adjoint": got1, "oracle_complex_step": ref1,
                         "rel_diff": abs(got1 - ref1) / max(abs(ref1), 1e-300),
                         "oracle_s": time.perf_counter() - t0})
    aflops = adjoint_flop_model(mech, M) * n * nsteps
    achieved = aflops / t_b / 1e12
    return {"workload": "adjoint: 4096 cells, 100 species / 500 reactions, 50 fixed ROK4E steps of 1e-7 s, "
                        "M=4; gradient of sum_c T_c(final) w.r.t. all 500 ln A_j",
            "value": n * nsteps / (t_f + t_b), "unit": "cell-steps/s (forward with checkpoints + adjoint)",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK, "traffic": None,
                         "kernel": "rok4e_adjoint_kernel<8>",
                         "algorithmic_tflop": aflops / 1e12,
                         "model": "bench.py adjoint_flop_model: value and dual right-hand-side passes and their "
                                  "reverse per step, Krylov and stage algebra"},
            "forward_s": t_f, "adjoint_s": t_b, "reps": len(tf), "adjoint_lanes_per_cell": sweep,
            "kernels": "rok4e_integrate_kernel (fixed steps), rok4e_adjoint_kernel, adjoint_reduce_kernel",
            "gradient_check": {
                "direction": "random unit vector in ln A (seed 7)",
                "vs_central_fd_h1e-6": {"cells": int(conv.sum()),
                                        "cells_rule": "central differences at h = 1e-6 and 1e-7 agree to 1e-3",
                                        "adjoint": got_s, "central_fd": fd_s,
                                        "rel_diff": abs(got_s - fd_s) / max(abs(fd_s), 1e-300)},
                "vs_oracle_complex_step": cs_cells}}


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The C oracle (gcc -O3, OpenMP over cells) on every host core, on a
    bounded sample of the headline workload: per step a fresh set of cells of
    the field (golden-ratio sequence), first integrated over dt from h0 = dt
    (untimed: it gives each cell its carried step, as the GPU arm's earlier
    step does), then timed over dt from that carried step."""
    if rank != 0:
        return 0
    from oracle import c_oracle
    from synth.fields import WORKLOADS, mechanism_for

    w = WORKLOADS["batched"]
    mech = mechanism_for(w)
    U = batched_field(w, 0)
    n = U.shape[0]
    M = w.krylov_dim
    co = c_oracle.COracle(mech)
    procs = max(1, os.cpu_count() or 1)
    per_step = args.ref_cells * procs

    def one(offset):
        Us = U[golden_cells(n, per_step, offset=offset)]
        _, h, _ = co.integrate(Us, w.dt, w.rtol, w.atol, M, threads=procs)
        t0 = time.perf_counter()
        co.integrate(Us, w.dt, w.rtol, w.atol, M, h0=h, threads=procs)
        return time.perf_counter() - t0

    for k in range(args.warmup):
        one(1000 + 7919 * k)
    t_total = sum(one(101 + 7919 * k) for k in range(args.steps))
    value = per_step * args.steps / t_total
    line = {
        "impl": "reference", "metric": "cell-steps/s", "value": value, "unit": "cell-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
        "config": {"workload": "batched: 2^20 constant-pressure cells per GPU from a 128^3 Gaussian random "
                               "temperature field (mean 1400 K, std 300 K), 53 species / 325 reactions, one "
                               "ROK4E reaction step of 1e-6 s per cell, rtol 1e-6, atol 1e-10",
                   "oracle_sample": f"{per_step} cells per step through the C oracle on {procs} host threads"},
        "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": procs, "kind": "oracle",
                         "sample": f"{per_step} cells per step (golden-ratio sequence over the field) x "
                                   f"{args.steps} steps, each over dt from its carried step"},
        "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- profiling cases
def run_plain(args):
    """Untimed split steps of the flame1d workload, or (--workload batched)
    one integration of the first --plain-cells cells of the batched field: the
    small cases used for ncu captures."""
    import torch

    import paper_1712_00953_gb300 as rk
    from synth.fields import WORKLOADS, field_tanh_front, mechanism_for

    if args.workload == "adjoint":
        from synth.fields import initial_state

        w = WORKLOADS["adjoint"]
        m = rk.mech_load(mechanism_for(w))
        U = torch.tensor(initial_state(w)[: args.plain_cells], device="cuda")
        n, N = U.shape
        ck = torch.empty(w.n_steps + 1, n, N, dtype=torch.float64, device="cuda")
        rk.rok4e_fixed_steps(m, U, w.dt, w.n_steps, w.krylov_dim, checkpoints=ck)
        ubar = torch.zeros_like(U)
        ubar[:, -1] = 1.0
        for _ in range(max(1, args.plain_steps)):
            grad, _ = rk.rok4e_adjoint(m, ck, ubar, w.dt, w.n_steps, w.krylov_dim, lanes_per_cell=args.lanes)
        torch.cuda.synchronize()
        print(json.dumps({"plain_steps": args.plain_steps, "cells": n, "grad_max": float(grad.abs().max())}))
        return 0
    if args.workload == "batched":
        w = WORKLOADS["batched"]
        m = rk.mech_load(mechanism_for(w))
        U = torch.tensor(batched_field(w, 0)[: args.plain_cells], device="cuda")
        hc = torch.zeros(U.shape[0], dtype=torch.float64, device="cuda")
        for _ in range(args.plain_steps):
            Y = U.clone()
            rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, args.krylov or w.krylov_dim, h_cell=hc,
                               opts=rk.Opts(cells_per_block=args.cells_per_block, lanes_per_cell=args.lanes,
                                            precision=PREC[args.precision]))
        torch.cuda.synchronize()
        print(json.dumps({"plain_steps": args.plain_steps, "cells": int(U.shape[0]), "T_max": float(Y[:, -1].max())}))
        return 0
    w = WORKLOADS["flame1d"]
    m = rk.mech_load(mechanism_for(w))
    _, U0 = field_tanh_front(w.n_cells, w.n_species, w.field_seed)
    U = torch.tensor(U0, device="cuda")
    hc = torch.zeros(U.shape[0], dtype=torch.float64, device="cuda")
    for _ in range(args.plain_steps):
        rk.simpler_split_step(m, U, w.dt, D_DIFF, LENGTH / U.shape[0], w.rtol, w.atol, w.krylov_dim, h_cell=hc,
                              opts=rk.Opts(lanes_per_cell=args.lanes, cells_per_block=args.flame_cells_per_block,
                                           precision=PREC[args.precision], queue_order=args.queue_order,
                                           blocks_per_sm=args.blocks_per_sm))
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
                 "fp64_warp_inst_1lane_4warps_per_sm", "df_fma", "i2f_f64"]
        print(json.dumps({"probes_ops_per_s": {nm: rk.probe_throughput(k) for k, nm in enumerate(names)}}))
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
    import dataclasses

    import torch

    import paper_1712_00953_gb300 as rk
    from synth.fields import WORKLOADS, initial_state, mechanism_for

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


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl", device_id=dev)
    line = run_headline(args, rank, world, dev, dist)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return 0
    if world == 1 and not args.headline_only:
        configs = {"small": run_small(args, dev), "flame1d": run_flame(args, dev, 0)}
        mixed = {}
        for name in ("mixed", "mixed-fp32jv", "mixed-df", "tensor", "exp32", "fp32jv"):
            mixed[name] = run_flame(args, dev, PREC[name], extras=False)
        mixed["note"] = ("the flame1d workload at each precision level against its FP64 value "
                         f"{configs['flame1d']['value']:.0f} cell-steps/s; accuracy against the FP64 oracle")
        configs["mixed"] = mixed
        cfg = line["config"]
        configs["mixed_batched"] = run_batched_levels(args, dev, cfg["krylov_dim"], args.lanes if args.no_autotune
                                                      else cfg["lanes_per_cell"], cfg["cells_per_block"])
        configs["adjoint"] = run_adjoint(args, dev)
        line["configs"] = configs
        line["gpu_launches"] += (configs["small"]["gpu_launches"] + configs["flame1d"]["gpu_launches"]
                                 + sum(v["gpu_launches"] for k, v in mixed.items() if k != "note"))
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--headline-only", action="store_true", help="skip the other workloads' blocks")
    ap.add_argument("--cpu-cells", type=int, default=64, help="C-oracle cells per host thread for the CPU baselines")
    ap.add_argument("--ref-cells", type=int, default=32, help="C-oracle cells per host thread per reference step")
    ap.add_argument("--e2e-steps", type=int, default=2, help="steps of the end-to-end measurement (headline)")
    ap.add_argument("--tune-cells", type=int, default=8192, help="autotuner sample of the batched field")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--krylov", type=int, default=0, help="force the Krylov dimension (0: tuned / 4)")
    ap.add_argument("--adjoint-reps", type=int, default=3)
    ap.add_argument("--level-steps", type=int, default=1, help="timed steps per precision level (2^18 cells)")
    ap.add_argument("--plain-steps", type=int, default=0,
                    help="run this many untimed steps and exit (profiling case)")
    ap.add_argument("--plain-cells", type=int, default=1 << 18, help="cells of the batched profiling case")
    ap.add_argument("--lanes", type=int, default=0, help="lanes per cell (0: library default)")
    ap.add_argument("--cells-per-block", type=int, default=0, help="cells per block, batched (0: library default)")
    ap.add_argument("--flame-cells-per-block", type=int, default=8, help="cells per block, flame1d")
    ap.add_argument("--precision", default="fp64", choices=list(PREC))
    ap.add_argument("--queue-order", type=int, default=3,
                    help="0 auto, 1 interleaved, 2 longest first, 3 static balanced bins")
    ap.add_argument("--unit-costs", action="store_true",
                    help="small RHS / J v / integration launches (for ncu instruction counts) and the probes")
    ap.add_argument("--skip-probes", action="store_true")
    ap.add_argument("--only", default="", choices=["", "adjoint", "flame1d", "small", "mixed_batched", "mixed"],
                    help="run one workload's block alone and print it (no headline line)")
    ap.add_argument("--study-kcap", type=float, default=0.0,
                    help="efficiency study on a variant of the batched mechanism with this cap on k C (1/s)")
    ap.add_argument("--study", default="", choices=["", "efficiency"],
                    help="efficiency: the ROK4E M / J v mode / explicit RK comparison over h_CFL")
    ap.add_argument("--workload", default="batched", choices=["batched", "flame1d", "adjoint"],
                    help="profiling case of --plain-steps")
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
    if args.only:
        import torch

        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        block = {"adjoint": lambda: run_adjoint(args, dev), "flame1d": lambda: run_flame(args, dev, 0),
                 "small": lambda: run_small(args, dev),
                 "mixed_batched": lambda: run_batched_levels(args, dev, 4, 32, 0),
                 "mixed": lambda: {name: run_flame(args, dev, PREC[name], extras=name == "fp64")
                                   for name in PREC}}[args.only]()
        print(json.dumps({"only": args.only, args.only: block}))
        return 0
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
