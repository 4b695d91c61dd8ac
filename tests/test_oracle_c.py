"""Pins of the C oracle (oracle/c/rok4e_oracle.c) -- CPU only.

The C oracle restates the method in compiled C for the long checks and the
timed CPU baseline.  It is pinned here against the numpy oracle -- an
independent implementation whose own pins tie it to the paper (order
conditions, convergence order, full-Krylov ROW equality, conservation, the
splitting recurrences) -- and against invariants directly:
* the right-hand side and its Jacobian-vector products (the C oracle's come
  from the complex step, the numpy oracle's from its analytic Jacobian) on
  all four mechanisms, at temperatures spanning both NASA ranges;
* whole adaptive integrations: the same accepted and rejected step counts and
  states to rounding, free running and replaying the numpy oracle's steps;
* Simpler split steps of the 1-D flame;
* element conservation over an integration, and a cell with f = 0 staying put.
"""

import numpy as np
import pytest

from oracle import c_oracle
from oracle import rok4e as orok
from oracle import splitting as osp
from oracle.kinetics import Kinetics, element_totals
from synth.fields import WORKLOADS, field_tanh_front, field_uniform, mechanism_for

P = 101325.0


@pytest.fixture(scope="module", autouse=True)
def built():
    c_oracle.build()


@pytest.mark.parametrize("name", ["small", "flame1d", "batched", "adjoint"])
def test_rhs_and_jvp_match_numpy_oracle(name):
    mech = mechanism_for(WORKLOADS[name])
    kin, co = Kinetics(mech), c_oracle.COracle(mech)
    U = field_uniform(12, mech.n_species, 3, 400.0, 2800.0)
    rng = np.random.default_rng(1)
    for u in U:
        f1, f2 = kin.rhs(u, P), co.rhs(u, P)
        assert np.max(np.abs(f1 - f2)) <= 1e-12 * np.max(np.abs(f1))
        v = rng.normal(size=u.shape)
        j1, j2 = kin.jvp(u, P, v), co.jvp(u, v, P, 0)
        assert np.max(np.abs(j1 - j2)) <= 1e-10 * np.max(np.abs(j1))
        jf, jf_ref = co.jvp(u, v, P, 1), kin.jvp_fd(u, P, v)  # the same forward difference on both sides
        assert np.max(np.abs(jf - jf_ref)) <= 1e-6 * np.max(np.abs(jf_ref))


@pytest.mark.parametrize("name,M", [("small", 4), ("flame1d", 4), ("flame1d", 6), ("batched", 4), ("batched", 8)])
def test_integration_matches_numpy_oracle(name, M):
    w = WORKLOADS[name]
    mech = mechanism_for(w)
    kin, co = Kinetics(mech), c_oracle.COracle(mech)
    U = field_uniform(6, mech.n_species, 5, 1000.0, 1800.0)
    ref, infos = orok.integrate_cells(kin, U, P, w.dt, w.rtol, w.atol, M, record=True)
    out, h, st = co.integrate(U, w.dt, w.rtol, w.atol, M)
    ns = mech.n_species
    assert [i["n_accept"] for i in infos] == st[:, 0].tolist()
    assert [i["n_reject"] for i in infos] == st[:, 1].tolist()
    assert np.all(st[:, 3] == 0)
    assert np.max(np.abs(out[:, :ns] - ref[:, :ns])) <= 1e-13
    assert np.max(np.abs(out[:, ns] - ref[:, ns])) <= 1e-9
    cap = max(len(i["trace"]) for i in infos) + 1
    rp = np.zeros((U.shape[0], cap))
    for c, i in enumerate(infos):
        for a, (hh, acc) in enumerate(i["trace"]):
            rp[c, a] = hh if acc else -hh
    out2, _, _ = co.integrate(U, w.dt, w.rtol, w.atol, M, replay=rp)
    assert np.max(np.abs(out2[:, :ns] - ref[:, :ns])) <= 1e-13
    assert np.max(np.abs(out2[:, ns] - ref[:, ns])) <= 1e-9


def test_simpler_split_steps_match_numpy_oracle():
    w = WORKLOADS["flame1d"]
    mech = mechanism_for(w)
    kin, co = Kinetics(mech), c_oracle.COracle(mech)
    npts = 24
    _, U = field_tanh_front(npts, mech.n_species, w.field_seed)
    dx = 1e-2 / npts
    Uo, h = U.copy(), np.zeros(npts)
    for _ in range(2):
        Uo, h, _, _ = osp.simpler_split_step_1d(kin, Uo, P, w.dt, 1e-4, dx, w.rtol, w.atol, 4, h_cell=h)
    Uc, hc, st = co.simpler_steps(U, np.zeros(npts), 2, w.dt, 1e-4, dx, w.rtol, w.atol, 4)
    ns = mech.n_species
    assert np.max(np.abs(Uc[:, :ns] - Uo[:, :ns])) <= 1e-13
    assert np.max(np.abs(Uc[:, ns] - Uo[:, ns])) <= 1e-9
    assert np.max(np.abs(hc - h) / h) <= 1e-5  # steps proposed from the error estimate (rounding-sensitive)


def test_conservation_and_steady_state():
    w = WORKLOADS["batched"]
    mech = mechanism_for(w)
    co = c_oracle.COracle(mech)
    U = field_uniform(8, mech.n_species, 9, 1200.0, 2200.0)
    out, _, st = co.integrate(U, w.dt, w.rtol, w.atol, 4)
    ns = mech.n_species
    e0, e1 = element_totals(mech, U[:, :ns]), element_totals(mech, out[:, :ns])
    assert np.max(np.abs(e1 - e0)) <= 1e-12 * np.max(np.abs(e0))
    assert np.max(np.abs(out[:, :ns].sum(axis=1) - U[:, :ns].sum(axis=1))) <= 1e-13
    # a balancing source -f(u) makes f + src exactly zero: the cell stays put
    src = -np.array([co.rhs(u, P) for u in U])
    out, _, st = co.integrate(U, w.dt, w.rtol, w.atol, 4, src=src)
    np.testing.assert_array_equal(out, U)
