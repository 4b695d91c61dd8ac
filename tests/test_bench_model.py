"""The roofline arithmetic of bench.py, on CPU.

`roofline.achieved` is algorithmic FP64 flops per launch divided by the
launch's time, with the flops from per-unit counts (bench.flop_model) times
the units the launch processed (bench.algorithmic_flops, from the per-cell
statistics the kernel returns).  These tests restate both from their stated
definitions with independent code (a dense net-coefficient matrix instead of
the per-reaction dictionaries, the unit counts from the ROK4E step's
structure: one Arnoldi process of M J v at the start and after every
accepted step but the last, two new right-hand sides per attempt and one per
fresh basis), so a drift in either side of the division fails here."""

import numpy as np
import pytest

import bench
from synth.fields import WORKLOADS, mechanism_for


def _net_nnz(mech):
    """Nonzero net stoichiometric coefficients, from a dense Nr x Ns matrix."""
    nu = np.zeros((mech.n_reactions, mech.n_species), dtype=np.int64)
    sp = np.asarray(mech.rxn_sp)
    cf = np.asarray(mech.rxn_nu)
    rows = np.repeat(np.arange(mech.n_reactions), sp.shape[1])
    keep = sp.reshape(-1) >= 0
    np.add.at(nu, (rows[keep], sp.reshape(-1)[keep]), cf.reshape(-1)[keep])
    return int(np.count_nonzero(nu))


def _model(mech, M):
    ns, nr = mech.n_species, mech.n_reactions
    N = ns + 1
    kind = np.asarray(mech.kind)
    tb, troe = int(np.sum(kind == 1)), int(np.sum(kind == 2))
    nnz = _net_nnz(mech)
    # right-hand side: 40 per species, 16 per reaction, 2 per net coefficient,
    # a third-body sum (2 per species) per pressure-dependent reaction, 40 per
    # Troe reaction, 10 cell scalars; exponentials: e^{+-g/RT} per species, one
    # per reaction, 7 per Troe reaction (4 exps, 2 logs, 1 exp) and ln T
    rhs = 40 * ns + 16 * nr + 2 * nnz + 2 * ns * (tb + troe) + 40 * troe + 10
    rhs_exp = 2 * ns + nr + 7 * troe + 1
    jvp = 25 * ns + 26 * nr + 2 * nnz + (2 * ns + 4) * (tb + troe) + 10
    # Arnoldi: f_n norm (3N), M normalisations and updates (5N each), CGS2's
    # two passes over the growing basis (4N flops per inner product and update
    # pair, twice, over 1 + 2 + ... + M columns)
    arnoldi = 3 * N + 5 * M * N + 2 * 4 * N * (M * (M + 1) // 2)
    # attempt: four stages of projection (Q^T F and Q c: 4MN) plus 6N of stage
    # sums, the two solutions and the error norm (22N), the M x M LU and the
    # correction matrix
    attempt = 4 * N * (4 * M + 6) + 22 * N + (2 * M ** 3) // 3 + 8 * M * M
    return dict(rhs=rhs, rhs_exp=rhs_exp, jvp=jvp, arnoldi=arnoldi, attempt=attempt)


@pytest.mark.parametrize("name", ["small", "flame1d", "batched", "adjoint"])
def test_flop_model_matches_its_definition(name):
    w = WORKLOADS[name]
    mech = mechanism_for(w)
    assert bench.flop_model(mech, w.krylov_dim) == _model(mech, w.krylov_dim)


def test_headline_unit_costs():
    # the per-unit figures quoted with the headline roofline (53 species, 325
    # reactions, M = 4): RHS 9,874 flops + 432 exps, J v 12,329, Arnoldi 5,562,
    # attempt 6,110; an accepted step (3 RHS, 4 J v, Arnoldi, 1 attempt) 116,530
    mech = mechanism_for(WORKLOADS["batched"])
    f = bench.flop_model(mech, 4)
    assert (f["rhs"], f["rhs_exp"], f["jvp"], f["arnoldi"], f["attempt"]) == (9874, 432, 12329, 5562, 6110)
    one_rhs = f["rhs"] + bench.EXP_FLOPS * f["rhs_exp"]
    assert one_rhs == 18514
    assert 3 * one_rhs + 4 * f["jvp"] + f["arnoldi"] + f["attempt"] == 116530


def test_algorithmic_flops_counts_units_per_cell():
    mech = mechanism_for(WORKLOADS["flame1d"])
    M = 4
    f = bench.flop_model(mech, M)
    rhs = f["rhs"] + bench.EXP_FLOPS * f["rhs_exp"]
    arn = M * f["jvp"] + f["arnoldi"]
    rng = np.random.default_rng(7)
    cells = []
    total = 0
    for _ in range(50):
        acc = int(rng.integers(0, 40))
        rej = int(rng.integers(0, 5))
        fresh = max(acc, 1)  # a basis at the start and after every accepted step but the last
        n_rhs = fresh + 2 * (acc + rej)
        cells.append((acc, rej, n_rhs, 0))
        total += n_rhs * rhs + fresh * arn + (acc + rej) * f["attempt"]
    st = np.array(cells, dtype=np.int32)
    assert bench.algorithmic_flops(f, st, M) == pytest.approx(float(total), rel=0, abs=0)
    # a cell that never accepted still built one basis
    assert bench.algorithmic_flops(f, np.array([[0, 3, 7, 2]], np.int32), M) == float(
        7 * rhs + arn + 3 * f["attempt"])


def test_adjoint_flop_model_is_linear_in_its_passes():
    # the adjoint of one step costs 3 value passes forward and back plus M dual
    # passes each way plus three times the step's Krylov algebra: doubling M
    # adds M dual passes each way and the larger Krylov algebra
    mech = mechanism_for(WORKLOADS["adjoint"])
    a4, a8 = bench.adjoint_flop_model(mech, 4), bench.adjoint_flop_model(mech, 8)
    f4, f8 = bench.flop_model(mech, 4), bench.flop_model(mech, 8)
    dual_pair = (a8 - 3 * (f8["arnoldi"] + f8["attempt"]) - (a4 - 3 * (f4["arnoldi"] + f4["attempt"]))) / 4
    # one dual forward plus one dual reverse pass is more than 2.5x a value
    # right-hand side with its exponentials, and less than 10x
    one_rhs = f4["rhs"] + bench.EXP_FLOPS * f4["rhs_exp"]
    assert 2.5 * f4["rhs"] < dual_pair < 10 * one_rhs
    assert a4 == pytest.approx(753398.0, rel=1e-12)  # 0.75 MFLOP per cell-step, as quoted
