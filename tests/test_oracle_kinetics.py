"""Pins of the oracle's kinetics (the 0-D reactor source of Eq. cv_reactor, read
as a constant-pressure reactor with textbook gas kinetics).

Each pin checks a property fixed by physics or mathematics rather than a
retyped formula: conservation of mass, elements and enthalpy; thermodynamic
consistency (cp = dh/dT, ds/dT = cp/T, continuity at T_mid, van 't Hoff);
detailed balance at equilibrium; the mass-action law for a known rate
constant; Lindemann / Troe limits; linearity in the third-body concentration;
and the analytic Jacobian against complex-step differentiation.
"""

import numpy as np
import pytest

from oracle.kinetics import R_GAS, Kinetics, element_totals
from synth.fields import WORKLOADS, initial_state, mechanism_for
from synth.mechanism import ELEMENT_MASS, single_reaction_mechanism

P = 101325.0


@pytest.fixture(scope="module", params=["small", "flame1d"])
def case(request):
    w = WORKLOADS[request.param]
    mech = mechanism_for(w)
    return mech, Kinetics(mech), initial_state(w)


def _sample(U, n=5):
    return U[np.linspace(0, len(U) - 1, n).astype(int)]


def test_mass_and_element_conservation_of_rhs(case):
    mech, kin, U = case
    ns = mech.n_species
    for u in _sample(U):
        f = kin.rhs(u, P)
        scale = np.max(np.abs(f[:ns]))
        assert abs(f[:ns].sum()) < 1e-13 * scale
        de = element_totals(mech, f[None, :ns])[0]
        assert np.max(np.abs(de)) < 1e-12 * scale / ELEMENT_MASS.min()


def test_enthalpy_is_conserved(case):
    # constant-pressure adiabatic: d/dt sum_k Y_k h_k / W_k = 0
    mech, kin, U = case
    ns = mech.n_species
    for u in _sample(U):
        f = kin.rhs(u, P)
        T = u[ns]
        cp_R, h_RT, _, _ = kin.thermo(T)
        h_mass = h_RT * R_GAS * T / mech.W
        cp_mass = np.sum(u[:ns] * cp_R * R_GAS / mech.W)
        dH = np.sum(h_mass * f[:ns]) + cp_mass * f[ns]
        assert abs(dH) < 1e-10 * np.sum(np.abs(h_mass * f[:ns]))


def test_thermo_consistency(case):
    mech, kin, _ = case
    for T in (350.0, 800.0, 1500.0, 2600.0):
        dT = 1e-3
        cp, hp, sp, dcp = kin.thermo(T + dT)
        cm, hm, sm, _ = kin.thermo(T - dT)
        c0, h0, s0, d0 = kin.thermo(T)
        # cp = dh/dT, ds/dT = cp/T, d(cp)/dT as returned
        assert np.allclose(((hp * (T + dT) - hm * (T - dT)) / (2 * dT)), c0, rtol=1e-7, atol=1e-7)
        assert np.allclose((sp - sm) / (2 * dT), c0 / T, rtol=1e-6, atol=1e-9)
        assert np.allclose((cp - cm) / (2 * dT), d0, rtol=1e-5, atol=1e-9)


def test_thermo_continuous_at_midpoint(case):
    mech, kin, _ = case
    for k in range(mech.n_species):
        tm = mech.nasa[k, 1]
        lo = [x[k] for x in kin.thermo(tm * (1 - 1e-12))]
        hi = [x[k] for x in kin.thermo(tm * (1 + 1e-12))]
        assert np.allclose(lo[:3], hi[:3], rtol=1e-8, atol=1e-8)


def test_thermo_range_is_chosen_by_t_mid(case):
    """NASA-7: below T_mid the low-temperature coefficients alone apply,
    above it the high-temperature ones alone: scrambling the set that does
    not apply leaves cp, h and s unchanged, scrambling the one that does
    changes them."""
    mech, kin, _ = case
    tm = mech.nasa[:, 1]
    rng = np.random.default_rng(14)
    for lo_side in (True, False):
        T = float(np.min(tm)) * 0.8 if lo_side else float(np.max(tm)) * 1.2
        other = mech.copy()
        same = mech.copy()
        cols_other = slice(10, 17) if lo_side else slice(3, 10)
        cols_same = slice(3, 10) if lo_side else slice(10, 17)
        other.nasa[:, cols_other] *= 1.0 + 0.1 * rng.normal(size=other.nasa[:, cols_other].shape)
        same.nasa[:, cols_same] *= 1.0 + 0.1 * rng.normal(size=same.nasa[:, cols_same].shape)
        ref = kin.thermo(T)[:3]
        for a, b in zip(Kinetics(other).thermo(T)[:3], ref):
            np.testing.assert_array_equal(a, b)
        assert not np.allclose(Kinetics(same).thermo(T)[0], ref[0], rtol=1e-6)


def test_van_t_hoff(case):
    mech, kin, U = case
    u = _sample(U, 1)[0].copy()
    for T in (700.0, 1400.0):
        u[-1] = T
        dT = 1e-4 * T
        up, um = u.copy(), u.copy()
        up[-1] += dT
        um[-1] -= dT
        lnKp = np.log(kin.state(up, P)["Kc"])
        lnKm = np.log(kin.state(um, P)["Kc"])
        st = kin.state(u, P)
        dlnK = (lnKp - lnKm) / (2 * dT)
        # d ln Kc / dT = (Delta H / RT - Delta nu) / T
        _, h_RT, _, _ = kin.thermo(T)
        expect = (kin.nu @ h_RT - kin.dnu) / T
        assert np.allclose(dlnK, expect, rtol=1e-6, atol=1e-10)
        assert np.allclose(st["dlnKc"], expect, rtol=1e-12, atol=1e-14)


def test_detailed_balance_at_equilibrium():
    # A + B <-> C : choose C_C so that C_C / (C_A C_B) = Kc, then q = 0
    mech = single_reaction_mechanism([0, 1], [2], [(0, 1, 1, 0), (0, 1, 0, 1), (0, 2, 1, 1)],
                                     1e12, 0.5, 4.0e4)
    kin = Kinetics(mech)
    T = 1300.0
    st = kin.state(np.array([0.3, 0.3, 0.4, T]), P)
    Kc = st["Kc"][0]
    ctot = P / (R_GAS * T)
    # mole fractions x_A = x_B = x, x_C = 1 - 2x with (1-2x)/(x^2 ctot) = Kc
    a, b, c = Kc * ctot, 2.0, -1.0
    x = (-b + np.sqrt(b * b - 4 * a * c)) / (2 * a)
    X = np.array([x, x, 1 - 2 * x])
    Y = X * mech.W / np.sum(X * mech.W)
    st = kin.state(np.append(Y, T), P)
    fwd = st["k"][0] * st["Pf"][0]
    assert abs(st["q"][0]) < 1e-11 * fwd


def test_mass_action_with_known_rate_constant():
    # irreversible A + B -> C with k = 1e13 cm^3/(mol s) = 1e7 m^3/(mol s)
    mech = single_reaction_mechanism([0, 1], [2], [(0, 1, 1, 0), (0, 1, 0, 1), (0, 2, 1, 1)],
                                     1e13, 0.0, 0.0, reversible=False)
    kin = Kinetics(mech)
    T = 1000.0
    Y = np.array([0.2, 0.5, 0.3])
    u = np.append(Y, T)
    f = kin.rhs(u, P)
    Wbar = 1.0 / np.sum(Y / mech.W)
    rho = P * Wbar / (R_GAS * T)  # ideal gas
    CA, CB = rho * Y[0] / mech.W[0], rho * Y[1] / mech.W[1]
    rate = 1e7 * CA * CB  # mol / (m^3 s)
    assert f[2] == pytest.approx(mech.W[2] * rate / rho, rel=1e-12)
    assert f[0] == pytest.approx(-mech.W[0] * rate / rho, rel=1e-12)


def test_arrhenius_activation_energy():
    # Arrhenius plot: d ln k / d(1/T) = -Ea/R - b T
    Ea, b = 8.0e4, 1.3
    mech = single_reaction_mechanism([0, 1], [2], [(0, 1, 1, 0), (0, 1, 0, 1), (0, 2, 1, 1)],
                                     1e11, b, Ea, reversible=False)
    kin = Kinetics(mech)
    T = 1200.0
    u = np.array([0.2, 0.5, 0.3, T])
    eps = 1e-4
    lk = []
    for TT in (T * (1 + eps), T * (1 - eps)):
        u2 = u.copy()
        u2[-1] = TT
        lk.append(np.log(kin.state(u2, P)["k"][0]))
    slope = (lk[0] - lk[1]) / (1 / (T * (1 + eps)) - 1 / (T * (1 - eps)))
    assert slope == pytest.approx(-Ea / R_GAS - b * T, rel=1e-6)


def _troe_mech(a, T3, T1, T2):
    mech = single_reaction_mechanism([0, 1], [2], [(0, 1, 1, 0), (0, 1, 0, 1), (0, 2, 1, 1)],
                                     1e13, 0.0, 0.0, reversible=False)
    mech.kind[:] = 2
    mech.falloff[0] = (1e16, 0.0, 0.0, a, T3, T1, T2)
    return mech


def test_lindemann_limit_of_troe():
    # Fcent = 1 (a = 1, T* huge, no T** term) -> F = 1 and k = kinf Pr/(1+Pr)
    kin = Kinetics(_troe_mech(1.0, 100.0, 1e30, 0.0))
    T = 1000.0
    u = np.array([0.2, 0.5, 0.3, T])
    st = kin.state(u, P)
    kinf = 1e13 * 1e-6
    k0 = 1e16 * 1e-12
    M = np.sum(st["C"])
    expect = kinf * (k0 * M / kinf) / (1 + k0 * M / kinf)
    assert st["k"][0] == pytest.approx(expect, rel=1e-12)


def test_troe_center_value():
    # at log10 Pr = -c the broadening factor equals Fcent
    a, T3, T1, T2 = 0.6, 200.0, 1500.0, 5000.0
    kin = Kinetics(_troe_mech(a, T3, T1, T2))
    T = 1100.0
    Fc = (1 - a) * np.exp(-T / T3) + a * np.exp(-T / T1) + np.exp(-T2 / T)
    c = -0.4 - 0.67 * np.log10(Fc)
    Pr = 10.0 ** (-c)
    F = kin._troe_F(T, np.array([Pr]))[0][0]
    assert F == pytest.approx(Fc, rel=1e-12)
    # and F -> 1 is approached from below in neither limit exactly: F(Pr) <= 1
    for pr in (1e-8, 1e-2, 1.0, 1e3, 1e9):
        assert kin._troe_F(T, np.array([pr]))[0][0] <= 1.0 + 1e-15


def test_troe_broadening_width():
    """F = sqrt(Fcent) where the broadening ratio (log Pr + c) / (n - d (log Pr + c))
    is +1 or -1, i.e. at log Pr + c = n / (1 + d) and -n / (1 - d), d = 0.14:
    two points at different distances on either side of the centre, which fix
    n and d (and the sign of d) where the centre value cannot."""
    a, T3, T1, T2 = 0.6, 200.0, 1500.0, 5000.0
    kin = Kinetics(_troe_mech(a, T3, T1, T2))
    T = 1100.0
    Fc = (1 - a) * np.exp(-T / T3) + a * np.exp(-T / T1) + np.exp(-T2 / T)
    c = -0.4 - 0.67 * np.log10(Fc)
    n = 0.75 - 1.27 * np.log10(Fc)
    for x in (n / 1.14, -n / 0.86):
        F = kin._troe_F(T, np.array([10.0 ** (x - c)]))[0][0]
        assert F == pytest.approx(np.sqrt(Fc), rel=1e-12)
    # the mirror image of the lower point is not a half-width point
    F = kin._troe_F(T, np.array([10.0 ** (n / 0.86 - c)]))[0][0]
    assert abs(F - np.sqrt(Fc)) > 1e-3 * np.sqrt(Fc)


def test_third_body_linear_in_efficiencies():
    w = WORKLOADS["flame1d"]
    mech = mechanism_for(w)
    kin = Kinetics(mech)
    u = initial_state(w)[1500]
    q1 = kin.rop(u, P)
    m2 = mech.copy()
    m2.eff = m2.eff * 2.0
    q2 = Kinetics(m2).rop(u, P)
    tb = mech.kind == 1
    el = mech.kind == 0
    assert np.allclose(q2[tb], 2 * q1[tb], rtol=1e-13)
    assert np.array_equal(q2[el], q1[el])


@pytest.mark.parametrize("name", ["small", "flame1d", "batched"])
def test_jacobian_matches_complex_step(name):
    w = WORKLOADS[name]
    mech = mechanism_for(w)
    kin = Kinetics(mech)
    if name == "batched":
        from synth.fields import field_gaussian3d
        U = field_gaussian3d(mech.n_species, w.field_seed, n=16, n_cells=64)
    else:
        U = initial_state(w)
    for u in _sample(U, 3):
        J = kin.jacobian(u, P)
        N = len(u)
        Jcs = np.empty_like(J)
        for i in range(N):
            s = max(1.0, abs(u[i]))
            du = np.zeros(N, complex)
            du[i] = 1e-30j * s
            Jcs[:, i] = np.imag(kin.rhs(u + du, P)) / (1e-30 * s)
        scale = np.max(np.abs(Jcs), axis=1, keepdims=True) + 1e-300
        assert np.max(np.abs(J - Jcs) / scale) < 1e-10


def test_fd_jvp_converges_to_analytic(case):
    mech, kin, U = case
    u = _sample(U, 1)[0]
    v = np.random.default_rng(0).normal(size=len(u))
    v /= np.linalg.norm(v)
    jv = kin.jvp(u, P, v)
    jfd = kin.jvp_fd(u, P, v)
    assert np.max(np.abs(jv - jfd)) < 1e-4 * np.max(np.abs(jv))


def test_constant_volume_conserves_internal_energy_and_mass():
    w = WORKLOADS["flame1d"]
    mech = mechanism_for(w)
    kin = Kinetics(mech, reactor="cv")
    ns = mech.n_species
    for u in _sample(initial_state(w)):
        rho = 0.3
        f = kin.rhs(u, rho)
        T = u[ns]
        cp_R, h_RT, _, _ = kin.thermo(T)
        e_mass = (h_RT - 1.0) * R_GAS * T / mech.W  # internal energy per unit mass of species k
        cv_mass = np.sum(u[:ns] * (cp_R - 1.0) * R_GAS / mech.W)
        dE = np.sum(e_mass * f[:ns]) + cv_mass * f[ns]
        assert abs(dE) < 1e-10 * np.sum(np.abs(e_mass * f[:ns]))
        assert abs(f[:ns].sum()) < 1e-13 * np.max(np.abs(f[:ns]))


def test_constant_volume_jacobian_matches_complex_step():
    w = WORKLOADS["flame1d"]
    kin = Kinetics(mechanism_for(w), reactor="cv")
    for u in _sample(initial_state(w), 3):
        rho = 0.25
        J = kin.jacobian(u, rho)
        N = len(u)
        Jcs = np.empty_like(J)
        for i in range(N):
            s = max(1.0, abs(u[i]))
            du = np.zeros(N, complex)
            du[i] = 1e-30j * s
            Jcs[:, i] = np.imag(kin.rhs(u + du, rho)) / (1e-30 * s)
        scale = np.max(np.abs(Jcs), axis=1, keepdims=True) + 1e-300
        assert np.max(np.abs(J - Jcs) / scale) < 1e-10


def test_constant_volume_and_pressure_agree_on_species_rates_at_equal_density():
    w = WORKLOADS["small"]
    mech = mechanism_for(w)
    cp, cv = Kinetics(mech), Kinetics(mech, reactor="cv")
    u = initial_state(w)[3]
    st = cp.state(u, P)
    a, b = cp.rhs(u, P), cv.rhs(u, st["rho"])
    ns = mech.n_species
    np.testing.assert_allclose(b[:ns], a[:ns], rtol=1e-12, atol=1e-12 * np.abs(a[:ns]).max())
