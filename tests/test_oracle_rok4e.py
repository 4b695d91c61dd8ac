"""Pins of the oracle's ROK4E integrator (Sec. 4.1-4.3, Algorithm 1).

* At full Krylov dimension M = N the projected Jacobian equals the exact one
  (Sec. 4.1), so one ROK4E attempt must equal a classical ROW step of the
  untransformed form Eq. s_stage_row solved with a dense LU -- a textbook
  routine independent of the oracle's transformed stages, Arnoldi and Woodbury
  solve.
* Fixed-step order 4 on a linear system against the matrix exponential, and
  the degradation to order 3 when M < p (the Krylov condition needs M >= p).
* Steady-state preservation (Def. steady_state_preserving): f(u) = 0 exactly
  leaves u unchanged bit for bit.
* Linear invariants (element totals, sum of Y) survive a full adaptive step.
"""

import numpy as np
import pytest
import scipy.linalg

from oracle import rok4e
from oracle.kinetics import Kinetics, element_totals
from synth.fields import WORKLOADS, initial_state, mechanism_for


def dense_row_step(f, J, u, h):
    """Classical ROW step, Eq. s_stage_row with the exact Jacobian (and the h on
    the A_n sum gamma_ij k_j term), solved with a dense linear solve."""
    g = rok4e.GAMMA
    A = np.eye(len(u)) - h * g * J
    ks = []
    for i in range(4):
        arg = u + h * sum((rok4e.ALPHA_IJ[i, j] * ks[j] for j in range(i)), np.zeros_like(u))
        rhs = f(arg) + h * J @ sum((rok4e.GAMMA_IJ[i, j] * ks[j] for j in range(i)), np.zeros_like(u))
        ks.append(np.linalg.solve(A, rhs))
    return (u + h * sum(rok4e.B[j] * ks[j] for j in range(4)),
            u + h * sum(rok4e.BHAT[j] * ks[j] for j in range(4)))


def _nonlinear_system(n, seed):
    rng = np.random.default_rng(seed)
    L = rng.normal(size=(n, n)) - 3 * np.eye(n)
    c = rng.normal(size=n)

    def f(u):
        return L @ u + c + 0.3 * np.sin(u) * u[::-1]

    def jac(u):
        J = L + 0.3 * np.diag(np.cos(u) * u[::-1])
        J = J + 0.3 * np.diag(np.sin(u))[:, ::-1]
        return J
    return f, jac


def test_nonlinear_system_jacobian_is_exact():
    f, jac = _nonlinear_system(7, 3)
    u = np.linspace(-1, 1, 7)
    J = jac(u)
    eps = 1e-7
    Jfd = np.column_stack([(f(u + eps * e) - f(u - eps * e)) / (2 * eps) for e in np.eye(7)])
    assert np.max(np.abs(J - Jfd)) < 1e-7


@pytest.mark.parametrize("n,h", [(6, 0.05), (9, 0.3), (12, 1.0)])
def test_full_krylov_dimension_equals_dense_row(n, h):
    f, jac = _nonlinear_system(n, n)
    u = np.random.default_rng(1).normal(size=n)
    fn = f(u)
    J = jac(u)
    Q, H = rok4e.arnoldi(lambda v: J @ v, fn, n)
    assert Q.shape[1] == n
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) < 1e-13
    assert np.max(np.abs(Q @ H @ Q.T - J)) < 1e-12 * np.max(np.abs(J))
    us, uh, nf = rok4e.attempt(f, u, fn, Q, H, h)
    ur, urh = dense_row_step(f, J, u, h)
    scale = np.max(np.abs(ur))
    assert np.max(np.abs(us - ur)) < 1e-13 * scale
    assert np.max(np.abs(uh - urh)) < 1e-13 * scale
    assert nf == 2  # stages 2 and 3; stage 4 reuses stage 3's f


def test_chemistry_full_krylov_equals_dense_row():
    w = WORKLOADS["small"]
    kin = Kinetics(mechanism_for(w))
    u = initial_state(w)[5]
    p = 101325.0
    f = lambda x: kin.rhs(x, p)
    J = kin.jacobian(u, p)
    N = len(u)
    fn = f(u)
    Q, H = rok4e.arnoldi(lambda v: J @ v, fn, N)
    h = 2e-9
    us, uh, _ = rok4e.attempt(f, u, fn, Q, H, h)
    ur, urh = dense_row_step(f, J, u, h)
    # (an early breakdown leaves an invariant subspace, on which the step is exact too)
    assert np.max(np.abs(us - ur) / (1e-10 + np.abs(ur))) < 1e-8


def _linear_problem(n=8, seed=5):
    rng = np.random.default_rng(seed)
    V = rng.normal(size=(n, n))
    lam = -np.logspace(-0.5, 1.0, n)
    L = V @ np.diag(lam) @ np.linalg.inv(V)
    c = rng.normal(size=n)
    u0 = rng.normal(size=n)
    return L, c, u0


def _fixed_step_error(M, n_steps, L, c, u0, T=1.0):
    f = lambda u: L @ u + c
    jv_at = lambda u: (lambda v: L @ v)
    u, info = rok4e.integrate(f, jv_at, u0, T, 1.0, 1.0, M, fixed_h=T / n_steps)
    assert info["n_accept"] == n_steps
    # exact: u(T) = e^{LT} u0 + L^{-1}(e^{LT} - I) c
    E = scipy.linalg.expm(L * T)
    exact = E @ u0 + np.linalg.solve(L, (E - np.eye(len(u0))) @ c)
    return np.max(np.abs(u - exact))


def _fitted_order(M, L, c, u0, steps=(16, 32, 64, 128, 256)):
    errs = np.array([_fixed_step_error(M, n, L, c, u0) for n in steps])
    return np.polyfit(np.log(1.0 / np.array(steps)), np.log(errs), 1)[0]  # err ~ h^p


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_order_four_on_linear_system(seed):
    L, c, u0 = _linear_problem(seed=seed)
    assert 3.7 < _fitted_order(4, L, c, u0) < 4.3
    assert 3.7 < _fitted_order(8, L, c, u0) < 4.3  # M = N: classical ROW


@pytest.mark.parametrize("seed", [5, 6])
def test_krylov_dimension_below_order_loses_order(seed):
    L, c, u0 = _linear_problem(seed=seed)
    assert 2.6 < _fitted_order(3, L, c, u0) < 3.3


def test_embedded_local_error_order():
    L, c, u0 = _linear_problem()
    f = lambda u: L @ u + c
    fn = f(u0)
    Q, H = rok4e.arnoldi(lambda v: L @ v, fn, 4)
    d = []
    for h in (0.02, 0.01):
        us, uh, _ = rok4e.attempt(f, u0, fn, Q, H, h)
        d.append(np.max(np.abs(uh - us)))
    # u* - u^ = O(h^4): halving h divides the estimate by ~16
    assert 12 < d[0] / d[1] < 20


def test_steady_state_is_preserved_bit_exact():
    w = WORKLOADS["small"]
    kin = Kinetics(mechanism_for(w))
    p = 101325.0
    for u in initial_state(w)[:4]:
        src = -kin.rhs(u, p)  # balancing source: f(u) = R(u) - R(u) = 0 exactly
        f, jv_at = rok4e.reactor(kin, p, src)
        assert np.all(f(u) == 0.0)
        out, info = rok4e.integrate(f, jv_at, u, w.dt, w.rtol, w.atol, 4)
        assert np.array_equal(out, u)
        assert info["n_accept"] == 1 and info["n_reject"] == 0


def test_linear_invariants_conserved():
    w = WORKLOADS["small"]
    mech = mechanism_for(w)
    kin = Kinetics(mech)
    p = 101325.0
    U = initial_state(w)[:6]
    out, infos = rok4e.integrate_cells(kin, U, p, w.dt, w.rtol, w.atol, 4)
    ns = mech.n_species
    e0 = element_totals(mech, U[:, :ns])
    e1 = element_totals(mech, out[:, :ns])
    assert np.max(np.abs(e1 - e0) / np.abs(e0).max()) < 1e-12
    assert np.max(np.abs(out[:, :ns].sum(1) - U[:, :ns].sum(1))) < 1e-13
    # and the state really moved
    assert np.max(np.abs(out - U)[:, :ns]) > 1e-4


def test_adaptive_error_control_tracks_tolerance():
    w = WORKLOADS["small"]
    kin = Kinetics(mechanism_for(w))
    p = 101325.0
    U = initial_state(w)[:3]
    ref, _ = rok4e.integrate_cells(kin, U, p, w.dt, 1e-11, 1e-15, 4)
    errs = []
    for rtol in (1e-4, 1e-6, 1e-8):
        out, _ = rok4e.integrate_cells(kin, U, p, w.dt, rtol, rtol * 1e-4, 4)
        errs.append(np.max(np.abs(out - ref) / (np.abs(ref) + 1e-6)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 1e-4


def test_fd_and_analytic_jacobian_vector_modes_agree():
    w = WORKLOADS["small"]
    kin = Kinetics(mechanism_for(w))
    p = 101325.0
    U = initial_state(w)[:3]
    a, _ = rok4e.integrate_cells(kin, U, p, w.dt, w.rtol, w.atol, 4, jv_mode="analytic")
    b, _ = rok4e.integrate_cells(kin, U, p, w.dt, w.rtol, w.atol, 4, jv_mode="fd")
    assert np.max(np.abs(a - b)[:, :-1]) < 1e-5
    assert np.max(np.abs(a - b)[:, -1]) < 1e-2


def test_replay_reproduces_free_run():
    w = WORKLOADS["small"]
    kin = Kinetics(mechanism_for(w))
    p = 101325.0
    U = initial_state(w)[:2]
    a, ia = rok4e.integrate_cells(kin, U, p, w.dt, w.rtol, w.atol, 4, record=True)
    b, ib = rok4e.integrate_cells(kin, U, p, w.dt, w.rtol, w.atol, 4, replay=[i["trace"] for i in ia])
    assert np.array_equal(a, b)


def test_arnoldi_breakdown_on_invariant_subspace():
    # J = diag with f in the span of two eigenvectors: K_M has dimension 2
    J = np.diag([-1.0, -2.0, -3.0, -4.0, -5.0])
    f = np.array([1.0, 1.0, 0.0, 0.0, 0.0])
    Q, H = rok4e.arnoldi(lambda v: J @ v, f, 4)
    assert Q.shape[1] == 2
    assert np.allclose(np.sort(np.linalg.eigvals(H).real), [-2.0, -1.0])


def test_zero_rhs_gives_empty_basis():
    Q, H = rok4e.arnoldi(lambda v: v, np.zeros(4), 4)
    assert Q.shape == (4, 0)


def test_error_norm_is_rms_over_all_components():
    """Reading R5 (the paper leaves the norm open): the root mean square over
    all N components.  A component with no error dilutes it by sqrt(N/(N+1)),
    which a max norm would not; one error at the tolerance in every component
    gives err = 1 whatever N."""
    rng = np.random.default_rng(11)
    u = rng.uniform(0.5, 2.0, 6)
    d = rng.normal(size=6) * 1e-7
    e6 = rok4e.error_norm(u, u + d, 1e-6, 1e-9)
    e7 = rok4e.error_norm(np.append(u, 1.0), np.append(u + d, 1.0), 1e-6, 1e-9)
    assert e7 == pytest.approx(e6 * np.sqrt(6 / 7), rel=1e-13)
    sc = 1e-9 + 1e-6 * u
    assert rok4e.error_norm(u, u + sc, 1e-6, 1e-9) == pytest.approx(1.0, rel=1e-9)  # (u + sc) - u rounds


def test_error_weights_use_the_propagated_solution():
    """Reading R5: the weights atol + rtol |u*| come from the propagated
    (order-4) solution u*, not the embedded one: with atol = 0 and u^ - u* =
    rtol u* in every component the error is exactly 1, while weights from u^
    would give 1 / (1 + rtol)."""
    rtol = 1e-3
    u_star = np.array([1.0, 100.0, 0.25])
    u_hat = u_star * (1 + rtol)
    assert rok4e.error_norm(u_star, u_hat, rtol, 0.0) == pytest.approx(1.0, rel=1e-12)
    assert abs(rok4e.error_norm(u_star, u_hat, rtol, 0.0) - 1 / (1 + rtol)) > 1e-4


def test_pi_controller_uses_the_last_accepted_error():
    """Sec. 4.3's PI controller, h* = h min(5, max(0.2, 0.8 err_n^(0.4/4) /
    err*^(0.7/4))), with err_n the error of the last accepted step (1 before
    the first, floored at 1e-10): every recorded attempt's step follows from
    the previous attempt's error and the last accepted one, clipped to the
    end of the interval, and the carried h_last is the last proposal."""
    w = WORKLOADS["small"]
    kin = Kinetics(mechanism_for(w))
    f, jv_at = rok4e.reactor(kin, 101325.0)
    u0 = initial_state(w)[5]
    t_end = 1e-5
    _, info = rok4e.integrate(f, jv_at, u0, t_end, 1e-8, 1e-12, 4, record=True)  # h0 = t_end
    tr, errs = info["trace"], info["errs"]
    assert len(tr) > 10 and any(not acc for _, acc in tr) and sum(acc for _, acc in tr) > 5
    t, err_n = 0.0, 1.0
    for i in range(len(tr)):
        h, acc = tr[i]
        e = max(errs[i], 1e-10)
        proposal = h * min(5.0, max(0.2, 0.8 * err_n**0.1 / e**0.175))
        if acc:
            t += h
            err_n = e
        if i + 1 < len(tr):
            assert tr[i + 1][0] == pytest.approx(min(proposal, t_end - t), rel=1e-12), i
    assert tr[-1][1] and info["h_last"] == pytest.approx(proposal, rel=1e-12)


def test_carried_step_is_the_controllers_proposal():
    """h_last, the step a cell carries into its next split step, is the
    controller's proposal after the last accepted step, not that step (which
    the end of the interval clips): on a smooth problem it is larger (1.47 times here; exactly 1 if the accepted step were carried)."""
    A = np.diag([-1.0, -2.0, -0.5])
    f = lambda u: A @ u
    _, info = rok4e.integrate(f, lambda u: (lambda v: A @ v), np.ones(3), 1.0, 1e-3, 1e-6, 3,
                              h0=0.01, record=True)
    last_accepted = [h for h, acc in info["trace"] if acc][-1]
    assert info["h_last"] > 1.2 * last_accepted


def test_fd_increment_stays_finite_at_the_zero_state():
    """The finite-difference increment d = sqrt(eps) (1 + ||u||) / ||v|| of the
    matrix-free product keeps its (1 + ...) so that u = 0 still has a step: on
    an affine right-hand side the product is A v there too."""
    rng = np.random.default_rng(13)
    A = rng.normal(size=(5, 5))
    c = rng.normal(size=5)

    class Affine:
        def rhs(self, u, p, src=None):
            return A @ u + c

    _, jv_at = rok4e.reactor(Affine(), 1.0, jv_mode="fd")
    v = rng.normal(size=5)
    assert np.allclose(jv_at(np.zeros(5))(v), A @ v, rtol=1e-6, atol=1e-6 * np.abs(A @ v).max())
