"""Pins of the explicit Dormand-Prince 5(4) oracle (the efficiency study's
explicit reference method, Sec. 4.4): the tableau's order conditions in exact
rational arithmetic over all rooted trees up to order 5, observed orders on a
linear system with a closed-form solution, first-same-as-last bookkeeping,
replay, and agreement with ROK4E on a chemistry cell at tight tolerances."""

from fractions import Fraction as Fr

import numpy as np
import pytest
import scipy.linalg

from oracle import explicit, rok4e
from oracle.kinetics import Kinetics
from synth.fields import WORKLOADS, initial_state, mechanism_for


def _trees(max_order):
    """All rooted trees up to max_order, as sorted tuples of child trees."""
    by_order = {1: [()]}
    for n in range(2, max_order + 1):
        found = set()

        def extend(rest, min_key, children):
            if rest == 0:
                found.add(tuple(sorted(children)))
                return
            for k in range(1, rest + 1):
                for t in by_order[k]:
                    key = (k, t)
                    if key < min_key:
                        continue
                    extend(rest - k, key, children + [t])

        extend(n - 1, (0, ()), [])
        by_order[n] = sorted(found)
    return by_order


def _order(t):
    return 1 + sum(_order(c) for c in t)


def _gamma(t):
    g = _order(t)
    for c in t:
        g *= _gamma(c)
    return g


def _phi(t, A):
    """Stage vector Phi_i(t) of the elementary weight, exact."""
    s = len(A)
    out = [Fr(1)] * s
    for c in t:
        pc = _phi(c, A)
        for i in range(s):
            out[i] *= sum((A[i][j] * pc[j] for j in range(len(A[i]))), Fr(0))
    return out


def _conditions(b, order):
    A = explicit.A_EXACT
    trees = _trees(order)
    bad = []
    n = 0
    for k in range(1, order + 1):
        for t in trees[k]:
            n += 1
            lhs = sum(bi * p for bi, p in zip(b, _phi(t, A)))
            if lhs != Fr(1, _gamma(t)):
                bad.append((t, lhs, Fr(1, _gamma(t))))
    return n, bad


def test_tree_count():
    trees = _trees(5)
    assert [len(trees[k]) for k in range(1, 6)] == [1, 1, 2, 4, 9]


def test_fifth_order_solution_satisfies_all_17_conditions():
    n, bad = _conditions(explicit.B_EXACT, 5)
    assert n == 17 and bad == []


def test_embedded_solution_is_order_four_not_five():
    n, bad = _conditions(explicit.BHAT_EXACT, 4)
    assert n == 8 and bad == []
    _, bad5 = _conditions(explicit.BHAT_EXACT, 5)
    assert len(bad5) > 0


def test_row_sums_and_first_same_as_last():
    for i, row in enumerate(explicit.A_EXACT):
        assert sum(row, Fr(0)) == explicit.C_EXACT[i]
    assert explicit.A_EXACT[6] == explicit.B_EXACT[:6] and explicit.B_EXACT[6] == 0


def _linear_problem(n=6, seed=3):
    rng = np.random.default_rng(seed)
    V = np.eye(n) + 0.3 * rng.normal(size=(n, n))  # well-conditioned, not normal
    L = V @ np.diag(-np.logspace(-0.5, 0.5, n)) @ np.linalg.inv(V)
    return L, rng.normal(size=n), rng.normal(size=n)


def _exact(L, c, u0, T):
    E = scipy.linalg.expm(L * T)
    return E @ u0 + np.linalg.solve(L, (E - np.eye(len(u0))) @ c)


@pytest.mark.parametrize("seed", [3, 4])
def test_order_five_on_linear_system(seed):
    L, c, u0 = _linear_problem(seed=seed)
    ex = _exact(L, c, u0, 1.0)
    steps = np.array([16, 32, 64, 128])
    errs = []
    for n in steps:
        u, info = explicit.integrate(lambda u: L @ u + c, u0, 1.0, 1.0, 1.0, fixed_h=1.0 / n)
        assert info["n_accept"] == n and info["n_f"] == 1 + 6 * n  # first same as last
        errs.append(np.max(np.abs(u - ex)))
    p = np.polyfit(np.log(1.0 / steps), np.log(errs), 1)[0]
    assert 4.7 < p < 5.4, p


def test_embedded_difference_scales_as_h5():
    L, c, u0 = _linear_problem()
    f = lambda u: L @ u + c
    d = []
    hs = np.array([0.2, 0.1, 0.05])
    for h in hs:
        u5, u4, _, _ = explicit.attempt(f, u0, f(u0), h)
        d.append(np.max(np.abs(u5 - u4)))
    p = np.polyfit(np.log(hs), np.log(d), 1)[0]
    assert 4.6 < p < 5.4, p


def test_adaptive_run_meets_tolerance_and_replays():
    L, c, u0 = _linear_problem()
    ex = _exact(L, c, u0, 2.0)
    u, info = explicit.integrate(lambda u: L @ u + c, u0, 2.0, 1e-8, 1e-10, record=True)
    assert info["status"] == explicit.STATUS_OK and abs(info["t"] - 2.0) < 1e-12
    assert np.max(np.abs(u - ex)) < 1e-6
    assert info["n_f"] == 1 + 6 * (info["n_accept"] + info["n_reject"])
    u2, _ = explicit.integrate(lambda u: L @ u + c, u0, 2.0, 1e-8, 1e-10, replay=info["trace"])
    assert np.array_equal(u, u2)


def test_stiff_linear_system_is_stability_limited():
    """u' = L u with eigenvalues down to -1e5 over t = 1: the explicit pair is
    held near its stability bound (|h lambda| <~ 3.3) however loose the
    tolerance, while ROK4E with the full Krylov space steps freely."""
    rng = np.random.default_rng(8)
    n = 5
    V = np.linalg.qr(rng.normal(size=(n, n)))[0]
    lam = -np.array([1.0, 2.0, 10.0, 1e3, 1e5])
    L = V @ np.diag(lam) @ V.T
    u0 = rng.normal(size=n)
    ue, ie = explicit.integrate(lambda u: L @ u, u0, 1.0, 1e-3, 1e-6)
    ur, ir = rok4e.integrate(lambda u: L @ u, lambda u: (lambda v: L @ v), u0, 1.0, 1e-3, 1e-6, n)
    attempts_e = ie["n_accept"] + ie["n_reject"]
    assert attempts_e > 1e5 / 3.4 * 0.5, attempts_e
    assert ir["n_accept"] + ir["n_reject"] < attempts_e / 100
    ex = scipy.linalg.expm(L) @ u0
    assert np.max(np.abs(ue - ex)) < 1e-2 and np.max(np.abs(ur - ex)) < 1e-2


def test_agrees_with_rok4e_on_a_chemistry_cell():
    w = WORKLOADS["small"]
    mech = mechanism_for(w)
    kin = Kinetics(mech)
    u0 = initial_state(w)[3]
    dt = 1e-5
    ue, ie = explicit.integrate(lambda u: kin.rhs(u, 101325.0), u0, dt, 1e-9, 1e-13)
    f, jv_at = rok4e.reactor(kin, 101325.0)
    ur, ir = rok4e.integrate(f, jv_at, u0, dt, 1e-9, 1e-13, 4)
    ns = mech.n_species
    assert ie["status"] == 0 and ir["status"] == 0
    assert np.max(np.abs(ue[:ns] - ur[:ns])) < 1e-8 and abs(ue[ns] - ur[ns]) < 1e-5


def test_controller_exponent_matches_the_pair_order():
    """The embedded difference of the 5(4) pair scales as h^5, so the
    controller's h* = 0.9 err^(-1/5) h must bring the next error to 0.9^5
    (unclipped factors): checked at err = 10 on the linear system with tight
    tolerances, where the asymptotic law holds to ~1 %.  An exponent of -1/4
    would land near 0.33."""
    L, c, u0 = _linear_problem()
    f = lambda u: L @ u + c

    def err(h):
        u5, u4, _, _ = explicit.attempt(f, u0, f(u0), h)
        return explicit.error_norm(u5, u4, 1e-13, 1e-13)

    lo, hi = 1e-4, 1.0
    for _ in range(60):  # bisection for err(h) = 10
        mid = np.sqrt(lo * hi)
        lo, hi = (lo, mid) if err(mid) > 10 else (mid, hi)
    e = err(lo)
    assert 9.0 < e <= 10.0
    assert err(lo * explicit.step_factor(e)) == pytest.approx(0.9**5, rel=0.05)


def test_error_norm_is_rms_with_weights_from_the_propagated_solution():
    """Reading R22: the RMS norm of ROK4E, weights atol + rtol |u5| from the
    propagated 5th-order solution: an error-free component dilutes it by
    sqrt(N/(N+1)) (a max norm would not), and u4 - u5 = rtol u5 with atol = 0
    gives exactly 1 (weights from u4 would give 1 / (1 + rtol))."""
    rng = np.random.default_rng(12)
    u = rng.uniform(0.5, 2.0, 5)
    d = rng.normal(size=5) * 1e-7
    e5 = explicit.error_norm(u, u + d, 1e-6, 1e-9)
    e6 = explicit.error_norm(np.append(u, 1.0), np.append(u + d, 1.0), 1e-6, 1e-9)
    assert e6 == pytest.approx(e5 * np.sqrt(5 / 6), rel=1e-13)
    rtol = 1e-3
    u5 = np.array([1.0, 100.0, 0.25])
    assert explicit.error_norm(u5, u5 * (1 + rtol), rtol, 0.0) == pytest.approx(1.0, rel=1e-12)
