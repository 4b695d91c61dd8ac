"""Launch-shape autotuner for rok4e_integrate.

``tune`` times candidate launch shapes -- lanes per cell (a warp integrates
32/lanes cells at once) and cells per block -- on a sample of the caller's
cells, and caches the fastest per (GPU, Ns, Nr, M, sample signature) in a JSON
file.  ``tune_krylov_and_shape`` also chooses the Krylov dimension: since M
changes the method's results, a dimension is admissible only while its
solution stays as close to a tight-tolerance reference as the default M = 4's
(or within the requested tolerance), and the fastest admissible (M, shape)
pair wins.  ``sweep_krylov`` reports timings over M.

Only timing and comparisons happen here: every candidate runs the library's
kernels through the C ABI on copies of the same cells.
"""

from __future__ import annotations

import json
import os
import time

import torch

from . import Opts, rok4e_integrate

CANDIDATES = [(32, 0), (32, 8), (16, 0), (16, 8), (8, 0), (8, 4)]
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "rok4e_autotune.json")


def _key(m, M, n_sample, tag):
    dev = torch.cuda.get_device_name()
    return f"{dev}|ns={m.n_species}|nr={m.n_reactions}|M={M}|n={n_sample}|{tag}"


def _time_once(m, Y0, dt, rtol, atol, M, opts, src, reps):
    best = float("inf")
    for _ in range(reps):
        Y = Y0.clone()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        rok4e_integrate(m, Y, dt, rtol, atol, M, src=src, opts=opts)
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune(m, Y, dt, rtol, atol, M=4, *, src=None, sample=None, reps=2, cache_path=DEFAULT_CACHE, tag="",
         candidates=CANDIDATES, verbose=False):
    """Return Opts with the fastest (lanes_per_cell, cells_per_block) for these cells.

    Y: [ncell, N] CUDA float64 cells (not modified); ``sample`` limits the timed
    cells to the first ``sample`` rows."""
    n = Y.shape[0] if sample is None else min(sample, Y.shape[0])
    key = _key(m, M, n, tag)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        lanes, cpb = cache[key]["lanes"], cache[key]["cells_per_block"]
        return Opts(lanes_per_cell=lanes, cells_per_block=cpb)
    Y0 = Y[:n].contiguous()
    s0 = None if src is None else src[:n].contiguous()
    results = []
    for lanes, cpb in candidates:
        ms = _time_once(m, Y0, dt, rtol, atol, M, Opts(lanes_per_cell=lanes, cells_per_block=cpb), s0, reps)
        results.append((ms, lanes, cpb))
        if verbose:
            print(f"autotune {key}: lanes={lanes} cells_per_block={cpb}: {ms:.3f} ms")
    ms, lanes, cpb = min(results)
    cache[key] = {"lanes": lanes, "cells_per_block": cpb, "ms": ms, "when": time.time(),
                  "all": [{"lanes": l, "cells_per_block": c, "ms": t} for t, l, c in results]}
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return Opts(lanes_per_cell=lanes, cells_per_block=cpb)


def sweep_krylov(m, Y, dt, rtol, atol, dims=(4, 5, 6, 8), *, src=None, opts=None, reps=2):
    """Timings (ms) of one integration of the same cells for each Krylov dimension."""
    return {M: _time_once(m, Y.contiguous(), dt, rtol, atol, M, opts or Opts(), src, reps) for M in dims}


SHAPES = ((32, 0), (16, 0), (8, 0))


def _run(m, Y0, dt, rtol, atol, M, opts, reps):
    """Best-of-reps time (ms) and the result of one integration of copies of Y0."""
    best, Y = float("inf"), None
    for _ in range(reps):
        Y = Y0.clone()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        rok4e_integrate(m, Y, dt, rtol, atol, M, opts=opts)
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best, Y


def tune_krylov_and_shape(m, Y, dt, rtol, atol, dims=(4, 5, 6, 8), shapes=SHAPES, *, precision=0, reps=2,
                          accuracy_factor=1.5, cache_path=DEFAULT_CACHE, tag="", verbose=False):
    """Choose the Krylov dimension and launch shape for these cells.

    Y: [n, N] CUDA float64 sample (not modified).  Accuracy constraint: every
    M in ``dims`` integrates the sample once; its error against a reference
    (M = 8 at rtol and atol 1e-4 times the requested ones) in the integrator's
    own norm, err_M = max over cells of the RMS of (Y_M - Y_ref) /
    (atol + rtol |Y_ref|), must satisfy err_M <= max(1, accuracy_factor *
    err_4).  Among the admissible dimensions and ``shapes`` (lanes_per_cell,
    cells_per_block) the fastest pair wins.  Returns a dict with the choice,
    the timing table and the errors; cached like ``tune``."""
    n = int(Y.shape[0])
    key = _key(m, "4-8", n, f"krylov+shape|prec={precision}|dt={dt}|rtol={rtol}|atol={atol}|{tag}")
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        return dict(cache[key], cached=True)
    Y0 = Y.contiguous()
    _, ref = _run(m, Y0, dt, rtol * 1e-4, atol * 1e-4, 8, Opts(precision=precision), 1)
    sc = atol + rtol * ref.abs()
    errs, table = {}, []
    for M in dims:
        for lanes, cpb in shapes:
            ms, Yr = _run(m, Y0, dt, rtol, atol, M, Opts(lanes_per_cell=lanes, cells_per_block=cpb,
                                                        precision=precision), reps)
            if M not in errs:
                errs[M] = float((((Yr - ref) / sc) ** 2).mean(dim=1).sqrt().max().item())
            table.append({"M": M, "lanes_per_cell": lanes, "cells_per_block": cpb, "ms": ms})
            if verbose:
                print(f"autotune {key}: M={M} lanes={lanes} cells_per_block={cpb}: {ms:.3f} ms, err {errs[M]:.3g}")
    base = errs.get(4, min(errs.values()))
    admissible = {M for M, e in errs.items() if e <= max(1.0, accuracy_factor * base)}
    best = min((t for t in table if t["M"] in admissible), key=lambda t: t["ms"])
    out = {"M": best["M"], "lanes_per_cell": best["lanes_per_cell"], "cells_per_block": best["cells_per_block"],
           "sample_cells": n, "ms": best["ms"], "table": table,
           "err_vs_tight_reference": {str(M): e for M, e in errs.items()},
           "admissible_M": sorted(admissible),
           "rule": "fastest (M, shape) with err_M <= max(1, %.1f err_4) against M=8 at 1e-4 x the tolerances"
                   % accuracy_factor, "when": time.time()}
    cache[key] = out
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return dict(out, cached=False)
