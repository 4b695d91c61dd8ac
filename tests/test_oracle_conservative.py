"""Pins of the auxiliary-temperature reaction system (Eq. chemical_source_balanced
with Eq. aux_t_equation): the constant-volume reactor as its source-free
special case, the energy identity that defines w_T (checked as an exact
directional derivative by complex step), and the auxiliary temperature
converging to the one recovered from the conservative variables."""

import numpy as np
import pytest

from oracle import conservative, rok4e
from oracle.kinetics import Kinetics
from synth.fields import WORKLOADS, initial_state, mechanism_for


def _setup(name="small", row=5, seed=0, with_src=True):
    w = WORKLOADS[name]
    mech = mechanism_for(w)
    aux = conservative.AuxTReactor(mech)
    u0 = initial_state(w)[row]
    ns = mech.n_species
    rng = np.random.default_rng(seed)
    rho = 0.35
    vel = rng.normal(size=3) * 30.0
    u = aux.state_from(u0[:ns], u0[ns], rho, vel)
    src = None
    if with_src:
        src = np.zeros(aux.N)
        src[:ns] = rng.normal(size=ns) * 1e-2 * rho
        src[ns + 1] = float(np.sum(src[:ns]))  # mass source consistent with the species sources
        src[ns + 2:ns + 5] = rng.normal(size=3) * 10.0
        src[ns + 5] = rng.normal() * 1e5
    return mech, aux, u, src


def test_source_free_case_is_the_constant_volume_reactor():
    mech, aux, u, _ = _setup(with_src=False)
    ns = mech.n_species
    rho = u[ns + 1]
    Y = u[:ns] / rho
    f = aux.rhs(u)
    g = Kinetics(mech, reactor="cv").rhs(np.concatenate([Y, [u[ns]]]), rho)
    assert np.allclose(f[:ns] / rho, g[:ns], rtol=1e-12, atol=1e-12 * np.max(np.abs(g[:ns])))
    assert f[ns] == pytest.approx(g[ns], rel=1e-12)
    assert np.all(f[ns + 1:] == 0.0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_energy_identity_along_the_flow(seed):
    """g(u) = rho e(T) + |rho u|^2 / (2 rho) - rho E is constant along f: its
    directional derivative (exact, by complex step) vanishes."""
    mech, aux, u, src = _setup(seed=seed)
    f = aux.rhs(u, src)
    ns = mech.n_species

    def g(x):
        rho = x[ns + 1]
        mom = x[ns + 2:ns + 5]
        return aux.internal_energy(x) + 0.5 * np.dot(mom, mom) / rho - x[ns + 5]

    eps = 1e-30
    dg = np.imag(g(u.astype(complex) + 1j * eps * f)) / eps
    # magnitude of the individual terms of the identity
    from oracle.kinetics import R_GAS
    _, h_RT, _, _ = aux.kin.thermo(u[ns])
    e = (h_RT - 1.0) * R_GAS * u[ns] / aux.W
    vel = u[ns + 2:ns + 5] / u[ns + 1]
    scale = (np.sum(np.abs(e * f[:ns])) + abs(f[ns + 5]) + abs(np.dot(vel, f[ns + 2:ns + 5]))
             + 0.5 * np.dot(vel, vel) * abs(f[ns + 1]))
    assert abs(dg) < 1e-12 * scale, (dg, scale)
    # flipping one momentum source moves the derivative by exactly -2 u_x f_x
    f_bad = f.copy()
    f_bad[ns + 2] = -f_bad[ns + 2]
    dg_bad = np.imag(g(u.astype(complex) + 1j * eps * f_bad)) / eps
    assert dg_bad == pytest.approx(-2.0 * vel[0] * f[ns + 2], rel=1e-6, abs=1e-12 * scale)


def test_auxiliary_temperature_converges_to_the_conservative_one():
    mech, aux, u, src = _setup(seed=1)
    ns = mech.n_species
    assert aux.T_conservative(u) == pytest.approx(u[ns], rel=1e-12)
    diffs = []
    for rtol in (1e-5, 1e-8):
        f, jv_at = conservative.reactor(aux, src)
        out, info = rok4e.integrate(f, jv_at, u, 2e-6, rtol, rtol * 1e-4, 4)
        assert info["status"] == 0
        diffs.append(abs(out[ns] - aux.T_conservative(out)))
    assert diffs[1] < diffs[0] / 30 or diffs[1] < 1e-9, diffs


def test_complex_step_jacobian_matches_central_differences():
    mech, aux, u, src = _setup(seed=2)
    J = aux.jacobian_with_src(u, src)
    rng = np.random.default_rng(4)
    v = rng.normal(size=aux.N) * np.maximum(np.abs(u), 1e-6)
    h = 1e-7
    fd = (aux.rhs(u + h * v, src) - aux.rhs(u - h * v, src)) / (2 * h)
    assert np.allclose(J @ v, fd, rtol=1e-5, atol=1e-7 * np.max(np.abs(fd)))
