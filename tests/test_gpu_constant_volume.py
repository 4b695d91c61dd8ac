"""GPU constant-volume reactor (Eq. cv_reactor) against the oracle."""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1712_00953_gb300 as rk

    return rk


def _case(name, n):
    from synth.fields import WORKLOADS, field_uniform, mechanism_for

    w = WORKLOADS[name]
    mech = mechanism_for(w)
    U = field_uniform(n, mech.n_species, 23, 800.0, 2400.0)
    rho = np.random.default_rng(4).uniform(0.1, 0.6, n)
    return w, mech, U, rho


@pytest.mark.parametrize("name", ["small", "flame1d"])
def test_cv_rhs_and_jvp_match_oracle(rk, name):
    from oracle.kinetics import Kinetics

    w, mech, U, rho = _case(name, 40)
    kin = Kinetics(mech, reactor="cv")
    m = rk.mech_load(mech)
    Ug, rg = torch.tensor(U, device="cuda"), torch.tensor(rho, device="cuda")
    out = rk.chem_rhs_cv(m, Ug, rg).cpu().numpy()
    ref = np.array([kin.rhs(u, r) for u, r in zip(U, rho)])
    assert np.max(np.abs(out - ref) / np.max(np.abs(ref), axis=1, keepdims=True)) < 1e-11
    V = np.random.default_rng(8).normal(size=U.shape)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    jv = rk.chem_jvp_cv(m, Ug, torch.tensor(V, device="cuda"), rg).cpu().numpy()
    jref = np.array([kin.jvp(u, r, v) for u, r, v in zip(U, rho, V)])
    assert np.max(np.abs(jv - jref) / np.max(np.abs(jref), axis=1, keepdims=True)) < 1e-10


def test_cv_integration_replays_oracle_and_conserves_energy(rk):
    from oracle import rok4e as orok
    from oracle.kinetics import R_GAS, Kinetics
    from synth.fields import WORKLOADS, initial_state, mechanism_for

    w = WORKLOADS["small"]
    mech = mechanism_for(w)
    U = initial_state(w)[::16]
    rho = np.full(U.shape[0], 0.25)
    m = rk.mech_load(mech)
    Y = torch.tensor(U, device="cuda")
    st = torch.zeros(U.shape[0], 4, dtype=torch.int32, device="cuda")
    tr = torch.zeros(U.shape[0], 8192, dtype=torch.float64, device="cuda")
    rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, 4, stats=st,
                       opts=rk.Opts(trace=tr, rho_cell=torch.tensor(rho, device="cuda")))
    torch.cuda.synchronize()
    out, st, tr = Y.cpu().numpy(), st.cpu().numpy(), tr.cpu().numpy()
    assert np.all(st[:, 3] == 0)
    kin = Kinetics(mech, reactor="cv")
    ref = []
    for i in range(U.shape[0]):
        f, jv_at = orok.reactor(kin, rho[i])
        r, _ = orok.integrate(f, jv_at, U[i], w.dt, w.rtol, w.atol, 4,
                              replay=[(abs(h), h > 0) for h in tr[i] if h != 0.0])
        ref.append(r)
    ref = np.array(ref)
    ns = mech.n_species
    assert np.all(np.abs(out[:, :ns] - ref[:, :ns]) <= 1e-8 + 1e-6 * np.abs(ref[:, :ns]))
    assert np.max(np.abs(out[:, ns] - ref[:, ns])) <= 1e-6

    def energy(V):  # mixture internal energy per unit mass, J/kg
        e = []
        for v in V:
            _, h_RT, _, _ = kin.thermo(v[ns])
            e.append(np.sum(v[:ns] * (h_RT - 1.0) * R_GAS * v[ns] / mech.W))
        return np.array(e)

    e0, e1 = energy(U), energy(out)
    assert np.max(np.abs(e1 - e0) / np.abs(e0)) < 1e-8  # at the integrator's tolerance
    assert np.max(np.abs(out[:, ns] - U[:, ns])) > 1.0  # while the temperature moved
