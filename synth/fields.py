"""Seeded initial fields and the named workloads.

Each workload fixes a mechanism recipe, a field recipe and the integration
settings.  Sizes follow the five workloads this library is measured on:

``small``     10 species / 24 reactions, 256 cells, T ~ U(1000, 1500) K,
              one 1e-6 s step, M = 4, rtol 1e-6, atol 1e-10.
``flame1d``   1-D reaction-diffusion: 2048 points on 1 cm, 30 species / 150
              reactions (4 third-body, 2 Troe), tanh temperature front
              300 -> 2000 K, 1000 Simpler split steps of 1e-7 s.
``batched``   2^20 cells cut from a 128^3 Gaussian random temperature field
              (mean 1400 K, std 300 K), 53 species / 325 reactions, one 1e-6 s
              step, M = 4..8.
``mixed``     the ``flame1d`` field and mechanism, reduced-precision kernels.
``adjoint``   4096 cells, 100 species / 500 reactions, 50 fixed steps of 1e-7 s.

Mass fractions are Dirichlet(0.5) draws.  Pressure is 1 atm everywhere.
"""

from __future__ import annotations

import dataclasses

import numpy as np

from .mechanism import Mechanism, generate_mechanism

P_ATM = 101325.0


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n_species: int
    n_reactions: int
    n_third_body: int
    n_troe: int
    n_cells: int
    dt: float
    n_steps: int
    rtol: float
    atol: float
    krylov_dim: int
    mech_seed: int
    field_seed: int
    k_cap: float
    T_window: tuple
    fixed_step: bool = False
    split: bool = False


WORKLOADS = {
    "small": Workload("small", 10, 24, 0, 0, 256, 1e-6, 1, 1e-6, 1e-10, 4, 1001, 2001,
                      1.0e8, (900.0, 1600.0)),
    "flame1d": Workload("flame1d", 30, 150, 4, 2, 2048, 1e-7, 1000, 1e-6, 1e-10, 4, 1002, 2002,
                        1.0e8, (300.0, 2200.0), split=True),
    "batched": Workload("batched", 53, 325, 0, 0, 1 << 20, 1e-6, 1, 1e-6, 1e-10, 4, 1003, 2003,
                        1.0e8, (300.0, 3000.0)),
    "mixed": Workload("mixed", 30, 150, 4, 2, 2048, 1e-7, 1000, 1e-6, 1e-10, 4, 1002, 2002,
                      1.0e8, (300.0, 2200.0), split=True),
    "adjoint": Workload("adjoint", 100, 500, 0, 0, 4096, 1e-7, 50, 1e-6, 1e-10, 4, 1005, 2005,
                        1.0e8, (900.0, 1600.0), fixed_step=True),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]


def mechanism_for(w: Workload) -> Mechanism:
    return generate_mechanism(w.n_species, w.n_reactions, seed=w.mech_seed,
                              n_third_body=w.n_third_body, n_troe=w.n_troe, k_cap=w.k_cap,
                              T_window=w.T_window)


def _dirichlet(rng, n, k, alpha=0.5):
    y = rng.dirichlet(np.full(k, alpha), size=n)
    return y


def field_uniform(n_cells: int, n_species: int, seed: int, T_lo=1000.0, T_hi=1500.0):
    """State rows (Y_1..Y_Ns, T) with T ~ U(T_lo, T_hi) and Y ~ Dirichlet(0.5)."""
    rng = np.random.default_rng(seed)
    u = np.empty((n_cells, n_species + 1))
    u[:, :n_species] = _dirichlet(rng, n_cells, n_species)
    u[:, n_species] = rng.uniform(T_lo, T_hi, n_cells)
    return u


def field_tanh_front(n_points: int, n_species: int, seed: int, length=1e-2, width=1e-3,
                     T_cold=300.0, T_hot=2000.0):
    """1-D front: T = mid + half*tanh((x - L/2)/width); Y blends two Dirichlet(0.5)
    compositions with the same tanh weight.  Returns (x, u) with cell centres x."""
    rng = np.random.default_rng(seed)
    x = (np.arange(n_points) + 0.5) * (length / n_points)
    w = 0.5 * (1.0 + np.tanh((x - 0.5 * length) / width))
    y_cold = _dirichlet(rng, 1, n_species)[0]
    y_hot = _dirichlet(rng, 1, n_species)[0]
    u = np.empty((n_points, n_species + 1))
    u[:, :n_species] = (1.0 - w)[:, None] * y_cold[None, :] + w[:, None] * y_hot[None, :]
    mid, half = 0.5 * (T_hot + T_cold), 0.5 * (T_hot - T_cold)
    u[:, n_species] = mid + half * np.tanh((x - 0.5 * length) / width)
    return x, u


def field_gaussian3d(n_species: int, seed: int, n=128, corr=8.0, mean=1400.0, std=300.0,
                     T_clip=(300.0, 3000.0), half=True, n_cells=None):
    """Gaussian random temperature field on an n^3 periodic grid, smoothed by a
    Gaussian filter of width ``corr`` cells (applied in Fourier space), rescaled
    to (mean, std) and clipped.  ``half`` keeps the z < n/2 slab (n^3/2 cells).
    Y ~ Dirichlet(0.5) per cell.  ``n_cells`` optionally truncates the cell list."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, n, n))
    k = np.fft.fftfreq(n)
    kx, ky, kz = np.meshgrid(k, k, np.fft.rfftfreq(n), indexing="ij")
    filt = np.exp(-2.0 * (np.pi * corr) ** 2 * (kx**2 + ky**2 + kz**2))
    s = np.fft.irfftn(np.fft.rfftn(g) * filt, s=(n, n, n), axes=(0, 1, 2))
    if half:
        s = s[:, :, : n // 2]
    t = s.reshape(-1)
    t = (t - t.mean()) / t.std() * std + mean
    t = np.clip(t, *T_clip)
    if n_cells is not None:
        t = t[:n_cells]
    ncell = t.shape[0]
    u = np.empty((ncell, n_species + 1))
    u[:, :n_species] = _dirichlet(rng, ncell, n_species)
    u[:, n_species] = t
    return u


def initial_state(w: Workload, n_cells: int | None = None):
    """Initial state rows for a workload (``n_cells`` takes a prefix)."""
    ns = w.n_species
    if w.name in ("flame1d", "mixed"):
        _, u = field_tanh_front(w.n_cells, ns, w.field_seed)
    elif w.name == "batched":
        u = field_gaussian3d(ns, w.field_seed, n_cells=n_cells)
    else:
        u = field_uniform(w.n_cells, ns, w.field_seed)
    if n_cells is not None:
        u = u[:n_cells]
    return np.ascontiguousarray(u)
