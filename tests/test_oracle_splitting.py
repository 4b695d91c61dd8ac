"""Pins of the oracle's splitting (Sec. 3) and the 1-D reaction-diffusion step.

* Scalar linear analysis: the two-substep schemes with exact sub-flows equal the
  recurrence u_{n+1} = R u_n - Q (a + b) with the closed forms; the printed
  limits (R -> I for h -> inf, the |B| -> inf limits, the 5.99 bound, the
  |B| > 3|A| criterion).
* Steady-state preservation (Def. steady_state_preserving) for the balanced
  methods and its failure for Strang with an O(h^3) one-step deviation.
* Scalar PSR (Eq. scalar_psr): turning points Da_E = 15.90, Da_I = 832.84.
* Second-order convergence of Simpler splitting.
* 1-D diffusion without chemistry: the Simpler step is second-order accurate
  against the exact solution of the semi-discrete diffusion equation.
"""

import os

import numpy as np
import pytest
import scipy.linalg
import scipy.optimize
from scipy.integrate import solve_ivp

from oracle import splitting as sp
from oracle.kinetics import Kinetics
from synth.mechanism import single_reaction_mechanism

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def _paper(name):
    for line in open(GOLDEN):
        if line.startswith(name + " ") or line.startswith(name + "\t"):
            return float(line.split()[1])
    raise KeyError(name)


def _linear(A, B, a, b):
    fT = sp.exact_linear_flow(A, a)
    fR = sp.exact_linear_flow(B, b)
    return fT, fR, (lambda u: A * u + a), (lambda u: B * u + b)


@pytest.mark.parametrize("A,B,h", [(-1.0, -7.0, 0.37), (-0.3, -40.0, 2.0), (-2.0, -0.5, 0.05)])
def test_simpler_recurrence_matches_two_substep_scheme(A, B, h):
    a, b = 0.4, -0.9
    fT, fR, Top, _ = _linear(A, B, a, b)
    step = lambda u: sp.simpler_step(u, h, Top, fT, fR)
    R, Q = sp.simpler_R_Q(A, B, h)
    for u in (0.0, 1.0, -2.5):
        assert step(u) == pytest.approx(R * u - Q * (a + b), rel=1e-13, abs=1e-14)


@pytest.mark.parametrize("A,B,h", [(-1.0, -7.0, 0.37), (-0.3, -40.0, 2.0)])
def test_simple_balanced_recurrence_matches_scheme(A, B, h):
    a, b = 0.4, -0.9
    fT, fR, Top, Rop = _linear(A, B, a, b)
    R, Q = sp.simple_R_Q(A, B, h)
    step = lambda u: sp.simple_balanced_step(u, h, Top, Rop, fT, fR, reaction_first=False)
    for u in (0.0, 1.0):
        assert step(u) == pytest.approx(R * u - Q * (a + b), rel=1e-13, abs=1e-14)
    # reaction first: the same map with A and B exchanged
    R2, Q2 = sp.simple_R_Q(B, A, h)
    step2 = lambda u: sp.simple_balanced_step(u, h, Top, Rop, fT, fR, reaction_first=True)
    for u in (0.0, 1.0):
        assert step2(u) == pytest.approx(R2 * u - Q2 * (a + b), rel=1e-13, abs=1e-14)


def test_simpler_limits():
    # h -> inf: R -> 1 (Eq. simpler_large_h)
    R, _ = sp.simpler_R_Q(-1.0, -5.0, 200.0)
    assert R == pytest.approx(1.0, abs=1e-12)
    # |B| -> inf: R -> 1 - alpha (the printed 1 - alpha^2 does not follow from R)
    A, h = -1.0, 0.8
    R, _ = sp.simpler_R_Q(A, -1e9, h)
    alpha = np.exp(A * h / 2)
    assert R == pytest.approx(1 - alpha, rel=1e-8)
    assert abs(R - (1 - alpha**2)) > 0.1
    # stable for all h > 0 with A, B < 0 (|R| < 1; R -> 1 only as h -> inf)
    for h in np.logspace(-3, 3, 61):
        for B in (-0.1, -1.0, -10.0, -1e4):
            R = sp.simpler_R_Q(-1.0, B, h)[0]
            assert abs(R) < 1.0 or (h > 30 and abs(R) <= 1.0)


def test_simple_balanced_limits():
    A = -1.0
    # h -> inf.  The printed R gives (1 - B/A)/2; Eq. simple_large_h prints
    # (I + A^-1 B)/2, a sign slip.  With the printed R the method is stable for
    # all h exactly when |B| < 3|A| (the text prints "|B| > 3|A|", which would
    # contradict its own remark that stiff B destabilises the method).
    for B in (-2.0, -5.0):
        R, _ = sp.simple_R_Q(A, B, 300.0)
        assert R == pytest.approx(0.5 * (1 - B / A), rel=1e-10)
    ratio = _paper("simple_balanced_ratio_bound")
    R, _ = sp.simple_R_Q(A, A * ratio * 0.99, 300.0)
    assert abs(R) < 1.0
    R, _ = sp.simple_R_Q(A, A * ratio * 1.01, 300.0)
    assert abs(R) > 1.0
    # |B| >> |A| (A -> 0 at fixed B h): R -> (1 + beta)(2 + B h)/4 and the |B| h < 5.99 bound
    h = 0.3
    for Bh in (1.0, 4.0, 5.5):
        B = -Bh / h
        lim = 0.25 * (1 + np.exp(B * h)) * (2 + B * h)
        Rbig, _ = sp.simple_R_Q(A * 1e-9, B, h)
        assert Rbig == pytest.approx(lim, rel=1e-6, abs=1e-9)
    x = scipy.optimize.brentq(lambda x: 0.25 * (1 + np.exp(-x)) * (2 - x) + 1, 3.0, 8.0)
    assert x == pytest.approx(_paper("simple_balanced_Bh_bound"), abs=0.005)


def test_steady_state_preservation():
    A, B, a, b = -1.0, -30.0, 0.4, 2.1
    fT, fR, Top, Rop = _linear(A, B, a, b)
    u_inf = -(a + b) / (A + B)
    for h in (0.01, 0.3, 5.0):
        assert sp.simpler_step(u_inf, h, Top, fT, fR) == pytest.approx(u_inf, rel=1e-14)
        assert sp.simple_balanced_step(u_inf, h, Top, Rop, fT, fR) == pytest.approx(u_inf, rel=1e-14)
    dev = [abs(sp.strang_step(u_inf, h, fT, fR) - u_inf) for h in (0.02, 0.01)]
    assert dev[0] > 1e-6
    assert 6.0 < dev[0] / dev[1] < 10.0  # O(h^3)


def test_scalar_psr_turning_points():
    T_in, T_ad, T_a = _paper("psr_T_in"), _paper("psr_T_ad"), _paper("psr_T_a")
    Da = lambda T: sp.psr_steady_Da(T, T_in, T_ad, T_a)
    dDa = lambda T: (Da(T * (1 + 1e-7)) - Da(T * (1 - 1e-7))) / (2e-7 * T)
    T_ign = scipy.optimize.brentq(dDa, 0.151, 0.4)  # local max of Da(T): ignition
    T_ext = scipy.optimize.brentq(dDa, 0.5, 1.1)  # local min: extinction
    assert Da(T_ign) == pytest.approx(_paper("psr_Da_ignition"), abs=0.01)
    assert Da(T_ext) == pytest.approx(_paper("psr_Da_extinction"), abs=0.01)


def _psr_flows(Da):
    def flow_R(T, dt, src):
        s = solve_ivp(lambda t, y: sp.psr_rhs_parts(y, Da)[0] + src, (0, dt), [T], rtol=1e-12,
                      atol=1e-14, method="LSODA")
        return s.y[0, -1]

    def flow_T(T, dt, src):
        s = solve_ivp(lambda t, y: sp.psr_rhs_parts(y, Da)[1] + src, (0, dt), [T], rtol=1e-12,
                      atol=1e-14, method="LSODA")
        return s.y[0, -1]
    return flow_T, flow_R


@pytest.mark.parametrize("case", ["extinction", "ignition"])
def test_near_limit_psr_strang_early_onset(case):
    """Sec. 3.5's near-limit cases of the scalar PSR: with a fixed splitting
    step, Strang splitting extinguishes (ignites) far too early, while simple
    and Simpler balanced splitting, which keep the steady states, follow the
    unsplit solution's slow passage to within a step or two."""
    Da = _paper(f"psr_Da_near_{case}")
    T0 = _paper(f"psr_T0_near_{case}")
    thr, t_end, h = (0.4, 2000.0, Da / 10) if case == "extinction" else (0.6, 4e5, Da / 2)
    hit = (lambda T: T < thr) if case == "extinction" else (lambda T: T > thr)
    ref = solve_ivp(lambda t, y: sum(sp.psr_rhs_parts(y, Da)), (0, t_end), [T0], rtol=1e-12, atol=1e-14,
                    method="LSODA", dense_output=True)
    ts = np.linspace(0, t_end, 200001)
    t_ref = ts[np.argmax(hit(ref.sol(ts)[0]))]
    flow_T, flow_R = _psr_flows(Da)
    Top = lambda T: sp.psr_rhs_parts(T, Da)[1]
    Rop = lambda T: sp.psr_rhs_parts(T, Da)[0]
    steps = {"strang": lambda T: sp.strang_step(T, h, flow_T, flow_R),
             "simpler": lambda T: sp.simpler_step(T, h, Top, flow_T, flow_R),
             "simple_balanced": lambda T: sp.simple_balanced_step(T, h, Top, Rop, flow_T, flow_R)}
    onset = {}
    for name, step in steps.items():
        T, t = T0, 0.0
        while t < t_end and not hit(T):
            T, t = step(T), t + h
        onset[name] = t
    print(f"{case}: unsplit {t_ref:.1f}, " + ", ".join(f"{k} {v:.1f}" for k, v in onset.items()))
    assert onset["strang"] < 0.7 * t_ref
    for name in ("simpler", "simple_balanced"):
        assert abs(onset[name] - t_ref) < 0.02 * t_ref


def test_simpler_second_order_on_scalar_psr():
    Da = 100.0
    T0, t_end = 0.6, 2.0
    flow_T, flow_R = _psr_flows(Da)
    Top = lambda T: sp.psr_rhs_parts(T, Da)[1]
    ref = solve_ivp(lambda t, y: sum(sp.psr_rhs_parts(y, Da)), (0, t_end), [T0], rtol=1e-12,
                    atol=1e-14, method="LSODA").y[0, -1]
    errs = []
    for n in (8, 16, 32):
        T = T0
        for _ in range(n):
            T = sp.simpler_step(T, t_end / n, Top, flow_T, flow_R)
        errs.append(abs(T - ref))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((slopes > 1.8) & (slopes < 2.3)), (errs, slopes)


def test_laplacian_exact_for_quadratics_and_conservative():
    n, dx = 20, 0.1
    x = (np.arange(n) + 0.5) * dx
    U = (3 * x**2 - x + 1.0)[:, None]
    L = sp.laplacian_neumann(U, dx)
    assert np.allclose(L[1:-1, 0], 6.0, rtol=1e-9)
    V = np.random.default_rng(0).normal(size=(n, 3))
    assert np.allclose(sp.laplacian_neumann(V, dx).sum(axis=0), 0.0, atol=1e-9)


def test_ssprk3_is_third_order():
    lam = -1.3
    errs = [abs(sp.ssprk3(np.array([1.0]), h, lambda v: lam * v)[0] - np.exp(lam * h)) for h in (0.1, 0.05)]
    assert 14.0 < errs[0] / errs[1] < 18.0  # local error O(h^4)


def _inert_mechanism():
    # one reaction with negligible rate: chemistry is effectively off
    return single_reaction_mechanism([0, 1], [2], [(0, 1, 1, 0), (0, 1, 0, 1), (0, 2, 1, 1)],
                                     1e-300, 0.0, 0.0, reversible=False)


def test_simpler_1d_diffusion_second_order():
    mech = _inert_mechanism()
    kin = Kinetics(mech)
    n, length, D = 32, 1e-2, 1e-4
    dx = length / n
    x = (np.arange(n) + 0.5) * dx
    U0 = np.empty((n, 4))
    U0[:, 0] = 0.2 + 0.1 * np.cos(np.pi * x / length)
    U0[:, 1] = 0.5
    U0[:, 2] = 1 - U0[:, 0] - U0[:, 1]
    U0[:, 3] = 1000.0 + 300.0 * np.cos(2 * np.pi * x / length)
    # exact semi-discrete solution: exp(t D L) U0 with the Neumann Laplacian matrix
    Lm = sp.laplacian_neumann(np.eye(n), dx)
    t_end = 4e-5
    exact = scipy.linalg.expm(t_end * D * Lm) @ U0
    errs = []
    for steps in (4, 8, 16):
        U = U0.copy()
        h = t_end / steps
        for _ in range(steps):
            U, _, infos, _ = sp.simpler_split_step_1d(kin, U, 101325.0, h, D, dx, 1e-8, 1e-12, 4)
        errs.append(np.max(np.abs(U[:, 3] - exact[:, 3])))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((slopes > 1.8) & (slopes < 2.4)), (errs, slopes)


@pytest.mark.parametrize("scheme", sp.SCHEMES)
def test_all_1d_schemes_second_order_without_chemistry(scheme):
    mech = _inert_mechanism()
    kin = Kinetics(mech)
    n, length, D = 24, 1e-2, 1e-4
    dx = length / n
    x = (np.arange(n) + 0.5) * dx
    U0 = np.empty((n, 4))
    U0[:, 0] = 0.2 + 0.1 * np.cos(np.pi * x / length)
    U0[:, 1] = 0.5
    U0[:, 2] = 1 - U0[:, 0] - U0[:, 1]
    U0[:, 3] = 1000.0 + 300.0 * np.cos(2 * np.pi * x / length)
    Lm = sp.laplacian_neumann(np.eye(n), dx)
    t_end = 4e-5
    exact = scipy.linalg.expm(t_end * D * Lm) @ U0
    errs = []
    for steps in (4, 8, 16):
        U = U0.copy()
        for _ in range(steps):
            U = sp.split_step_1d(kin, U, 101325.0, t_end / steps, D, dx, 1e-9, 1e-13, 4, scheme)
        errs.append(np.max(np.abs(U[:, 3] - exact[:, 3])))
    if scheme == "strang":
        # without chemistry Strang is transport alone: SSP-RK3 half steps, no splitting error
        assert max(errs) < 1e-8, errs
        return
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((slopes > 1.8) & (slopes < 2.5)), (scheme, errs, slopes)


def test_simpler_split_matches_dedicated_function():
    from synth.fields import WORKLOADS, field_tanh_front, mechanism_for

    w = WORKLOADS["flame1d"]
    mech = mechanism_for(w)
    kin = Kinetics(mech)
    _, U = field_tanh_front(8, mech.n_species, w.field_seed)
    a = sp.split_step_1d(kin, U, 101325.0, 1e-8, 1e-4, 1e-2 / 8, 1e-6, 1e-10, 4, "simpler")
    b, _, _, _ = sp.simpler_split_step_1d(kin, U, 101325.0, 1e-8, 1e-4, 1e-2 / 8, 1e-6, 1e-10, 4,
                                          h_cell=np.zeros(8))
    np.testing.assert_array_equal(a, b)


def test_reaction_windows_give_the_full_field_step_at_their_centres():
    """The one-step SSP-RK3 transport correction reaches three points, so a
    sampled point's split step needs the reaction sub-step only on the seven
    points around it (the full-size GPU parity test relies on this): with the
    step sequences replayed, the windowed step equals the full-field step
    exactly at the window centres, near the boundaries too, and not one point
    further out."""
    from synth.fields import WORKLOADS, field_tanh_front, mechanism_for

    w = WORKLOADS["flame1d"]
    mech = mechanism_for(w)
    kin = Kinetics(mech)
    npts = 40
    _, U = field_tanh_front(npts, mech.n_species, w.field_seed)
    dx, D, p = 1e-2 / npts, 1e-4, 101325.0
    full, _, infos, _ = sp.simpler_split_step_1d(kin, U, p, w.dt, D, dx, w.rtol, w.atol, 4, record=True)
    centres = [3, 17, 20, 36]
    cells = sorted({c + d for c in centres for d in range(-3, 4)})
    replay = [infos[c]["trace"] if c in cells else None for c in range(npts)]
    win, _, _, _ = sp.simpler_split_step_1d(kin, U, p, w.dt, D, dx, w.rtol, w.atol, 4, replay=replay, cells=cells)
    assert np.array_equal(win[centres], full[centres])
    assert not np.array_equal(win[15], full[15])  # two points from an uncomputed one


def test_laplacian_ends_are_zero_flux_walls():
    """Reading R18, zero-gradient ends: the first point does not see the last
    one (no wrap-around), and a linear profile U = a + b x on cell centres,
    whose interior fluxes are all b, gains b / dx in the first cell and loses
    it in the last, since nothing crosses the walls."""
    n, dx, b = 12, 0.25, 3.0
    x = (np.arange(n) + 0.5) * dx
    U = (2.0 + b * x)[:, None]
    L = sp.laplacian_neumann(U, dx)
    assert np.allclose(L[1:-1, 0], 0.0, atol=1e-12)
    assert L[0, 0] == pytest.approx(b / dx, rel=1e-12) and L[-1, 0] == pytest.approx(-b / dx, rel=1e-12)
    V = np.random.default_rng(2).normal(size=(n, 2))
    W = V.copy()
    W[-1] += 5.0
    assert np.array_equal(sp.laplacian_neumann(V, dx)[:-2], sp.laplacian_neumann(W, dx)[:-2])


@pytest.mark.parametrize("scheme", sp.SCHEMES)
def test_1d_schemes_are_the_generic_schemes(scheme):
    """Each branch of split_step_1d is the scheme function pinned on the scalar
    problems above (Strang, Eq. balanced, simple balanced reaction first,
    Eq. simpler_balanced), driven by the 1-D flows: one SSP-RK3 step for
    transport, ROK4E per cell for reaction with the first step carried over."""
    from oracle import rok4e
    from synth.fields import WORKLOADS, field_tanh_front, mechanism_for

    w = WORKLOADS["flame1d"]
    mech = mechanism_for(w)
    kin = Kinetics(mech)
    n, p, dt, D = 8, 101325.0, 1e-8, 1e-4
    dx = 1e-2 / n
    _, U = field_tanh_front(n, mech.n_species, w.field_seed)
    hc = np.zeros(n)

    def flow_T(V, t, c):
        return sp.ssprk3(V, t, lambda X: sp.diffusion_op(X, D, dx) + c)

    def flow_R(V, t, src):
        out = V.copy()
        for i in range(n):
            s = None if np.isscalar(src) and src == 0.0 else src[i]
            f, jv_at = rok4e.reactor(kin, p, s)
            out[i], inf = rok4e.integrate(f, jv_at, V[i], t, w.rtol, w.atol, 4, h0=hc[i])
            hc[i] = inf["h_last"]
        return out

    def T_op(V):
        return sp.diffusion_op(V, D, dx)

    def R_op(V):
        return np.array([kin.rhs(u, p) for u in V])

    generic = {
        "simpler": lambda: sp.simpler_step(U, dt, T_op, flow_T, flow_R),
        "strang": lambda: sp.strang_step(U, dt, flow_T, flow_R),
        "simple_balanced": lambda: sp.simple_balanced_step(U, dt, T_op, R_op, flow_T, flow_R, True),
        "simple_balanced_transport_first": lambda: sp.simple_balanced_step(U, dt, T_op, R_op, flow_T, flow_R,
                                                                           False),
    }[scheme]()
    dedicated = sp.split_step_1d(kin, U, p, dt, D, dx, w.rtol, w.atol, 4, scheme)
    np.testing.assert_array_equal(dedicated, generic)
