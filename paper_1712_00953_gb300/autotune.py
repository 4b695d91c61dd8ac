"""Launch-shape autotuner for rok4e_integrate.

Times candidate launch shapes -- lanes per cell (a warp integrates 32/lanes
cells at once) and cells per block -- on a sample of the caller's cells, and
caches the fastest per (GPU, Ns, Nr, M, sample signature) in a JSON file.  The
Krylov dimension is part of the key rather than a tuned knob because it changes
the method's results; ``sweep_krylov`` reports timings over M for a caller who
wants to choose it.

Only timing happens here: every candidate runs the library's kernels through
the C ABI on copies of the same cells.
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
