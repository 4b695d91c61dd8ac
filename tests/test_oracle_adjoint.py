"""Pins of the oracle's gradient of fixed-step ROK4E w.r.t. ln A and u0: the
complex-step derivative agrees with central finite differences (whose
truncation error is O(d^2)) on the sensitivities large enough for finite
differences to resolve, converges at that rate with a Richardson-extrapolated
limit equal to it to 1e-8, and is linear in the objective weights."""

import numpy as np
import pytest

from oracle import adjoint as oad
from oracle.kinetics import Kinetics
from synth.fields import WORKLOADS, field_uniform, mechanism_for

P = 101325.0


@pytest.fixture(scope="module")
def case():
    w = WORKLOADS["small"]
    mech = mechanism_for(w)
    u0 = field_uniform(1, mech.n_species, 11, 1000.0, 1500.0)[0]
    return Kinetics(mech), u0


def test_complex_step_matches_central_differences(case):
    kin, u0 = case
    h, n = 2e-8, 6
    js = np.arange(kin.nr)
    cs = oad.grad_complex_step(kin, u0, P, h, n, 4, js)
    big = np.argsort(-np.abs(cs))[:5]
    fd = oad.grad_central_fd(kin, u0, P, h, n, 4, big, d=1e-4)
    assert np.max(np.abs(fd - cs[big]) / np.abs(cs[big])) < 1e-4


def test_complex_step_is_the_limit_of_central_differences(case):
    """Central differences at d and d/2 converge to the complex-step value at
    the O(d^2) rate, and their Richardson extrapolation (O(d^4)) agrees with
    it to 1e-8 relative -- tight enough to see a 1e-6 error in the
    derivative itself."""
    kin, u0 = case
    h, n = 2e-8, 6
    js = np.arange(kin.nr)
    cs = oad.grad_complex_step(kin, u0, P, h, n, 4, js)
    big = np.argsort(-np.abs(cs))[:5]
    d = 1e-2
    f1 = oad.grad_central_fd(kin, u0, P, h, n, 4, big, d=d)
    f2 = oad.grad_central_fd(kin, u0, P, h, n, 4, big, d=d / 2)
    e1, e2 = np.abs(f1 - cs[big]), np.abs(f2 - cs[big])
    assert np.all((e1 / e2 > 3.5) & (e1 / e2 < 4.5))
    rich = (4.0 * f2 - f1) / 3.0
    assert np.max(np.abs(rich - cs[big]) / np.abs(cs[big])) < 1e-8


def test_gradient_is_linear_in_the_objective(case):
    kin, u0 = case
    h, n = 2e-8, 4
    js = [0, 5, 11]
    wT = np.zeros(len(u0))
    wT[-1] = 1.0
    wY = np.zeros(len(u0))
    wY[2] = 1.0
    a = oad.grad_complex_step(kin, u0, P, h, n, 4, js, weights=wT)
    b = oad.grad_complex_step(kin, u0, P, h, n, 4, js, weights=wY)
    c = oad.grad_complex_step(kin, u0, P, h, n, 4, js, weights=2.0 * wT - 3.0 * wY)
    np.testing.assert_allclose(c, 2.0 * a - 3.0 * b, rtol=1e-10, atol=1e-14 * np.abs(a).max())


def test_complex_step_final_state_equals_real_run(case):
    kin, u0 = case
    real = oad.final_state(kin, u0, P, 2e-8, 5, 4)
    cplx = oad.final_state(kin, u0.astype(complex), P, 2e-8, 5, 4, kin.lnA_input.astype(complex))
    np.testing.assert_allclose(np.real(cplx), real, rtol=1e-13, atol=1e-15)
    assert np.all(np.imag(cplx) == 0.0)
