"""GPU parity of the auxiliary-temperature reaction system (Eq.
chemical_source_balanced with Eq. aux_t_equation) against the FP64 oracle
(oracle/conservative.py): right-hand side, analytic and finite-difference
J v (the oracle's Jacobian is a complex-step derivative, independent of the
kernels' hand derivation), ROK4E and RKDP integrations replayed through the
oracle, the source-free constant-volume special case and an exact steady
state."""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

Y_ABS, Y_REL, T_ABS = 1e-8, 1e-6, 1e-6


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1712_00953_gb300 as rk

    return rk


def _cells(name, n, seed=0, with_src=True):
    from oracle.conservative import AuxTReactor
    from synth.fields import WORKLOADS, initial_state, mechanism_for

    w = WORKLOADS[name]
    mech = mechanism_for(w)
    aux = AuxTReactor(mech)
    ns = mech.n_species
    rng = np.random.default_rng(seed)
    base = initial_state(w)
    rows = base[np.linspace(0, base.shape[0] - 1, n).astype(int)]
    U = np.array([aux.state_from(r[:ns], r[ns], rng.uniform(0.2, 1.2), rng.normal(size=3) * 40.0) for r in rows])
    S = None
    if with_src:
        S = np.zeros_like(U)
        S[:, :ns] = rng.normal(size=(n, ns)) * 1e-2 * U[:, [ns + 1]]
        S[:, ns + 1] = S[:, :ns].sum(axis=1)
        S[:, ns + 2:ns + 5] = rng.normal(size=(n, 3)) * 10.0
        S[:, ns + 5] = rng.normal(size=n) * 1e5
    return w, mech, aux, U, S


def _t(x):
    return None if x is None else torch.tensor(x, device="cuda")


@pytest.mark.parametrize("name", ["small", "flame1d"])
def test_rhs_matches_oracle(rk, name):
    w, mech, aux, U, S = _cells(name, 48)
    m = rk.mech_load(mech)
    out = rk.chem_rhs_aux(m, _t(U), _t(S)).cpu().numpy()
    ref = np.array([aux.rhs(u, s) for u, s in zip(U, S)])
    ns = mech.n_species
    sc = np.max(np.abs(ref[:, :ns]), axis=1, keepdims=True)
    assert np.max(np.abs(out[:, :ns] - ref[:, :ns]) / sc) < 1e-11
    assert np.max(np.abs(out[:, ns] - ref[:, ns]) / np.abs(ref[:, ns])) < 1e-10
    assert np.array_equal(out[:, ns + 1:], S[:, ns + 1:])


@pytest.mark.parametrize("name", ["small", "flame1d"])
def test_jvp_matches_complex_step_jacobian(rk, name):
    w, mech, aux, U, S = _cells(name, 24, seed=1)
    m = rk.mech_load(mech)
    V = np.random.default_rng(3).normal(size=U.shape) * np.maximum(np.abs(U), 1e-8)
    out = rk.chem_jvp_aux(m, _t(U), _t(V), _t(S)).cpu().numpy()
    ref = np.array([aux.jacobian_with_src(u, s) @ v for u, s, v in zip(U, S, V)])
    sc = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.max(np.abs(out - ref) / sc) < 1e-9


def test_fd_jvp_matches_oracle_fd(rk):
    """Forward-difference J v (increment sqrt(eps)(1 + ||u||)/||v||, which the
    energy component dominates for conservative rows) against the oracle's
    same difference quotient."""
    from oracle.conservative import reactor

    w, mech, aux, U, S = _cells("small", 16, seed=2)
    m = rk.mech_load(mech)
    V = np.random.default_rng(5).normal(size=U.shape)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    f = rk.chem_jvp_aux(m, _t(U), _t(V), _t(S), mode=1).cpu().numpy()
    ref = np.array([reactor(aux, s, "fd")[1](u)(v) for u, s, v in zip(U, S, V)])
    sc = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.max(np.abs(f - ref) / sc) < 1e-4


def test_source_free_system_is_the_constant_volume_reactor(rk):
    w, mech, aux, U, _ = _cells("flame1d", 32, seed=4, with_src=False)
    m = rk.mech_load(mech)
    ns = mech.n_species
    out = rk.chem_rhs_aux(m, _t(U)).cpu().numpy()
    rho = U[:, ns + 1]
    Ycv = np.concatenate([U[:, :ns] / rho[:, None], U[:, [ns]]], axis=1)
    cv = rk.chem_rhs_cv(m, _t(Ycv), _t(rho)).cpu().numpy()
    sc = np.max(np.abs(cv[:, :ns]), axis=1, keepdims=True)
    assert np.max(np.abs(out[:, :ns] / rho[:, None] - cv[:, :ns]) / sc) < 1e-11
    assert np.max(np.abs(out[:, ns] - cv[:, ns]) / np.abs(cv[:, ns])) < 1e-10
    assert np.all(out[:, ns + 1:] == 0.0)


def _close(gpu, ref, ns, what):
    dY = np.abs(gpu[:, :ns] - ref[:, :ns])
    excess = dY - (Y_ABS * ref[:, [ns + 1]] + Y_REL * np.abs(ref[:, :ns]))
    dT = np.abs(gpu[:, ns] - ref[:, ns])
    assert np.all(excess <= 0.0), f"{what}: max excess {excess.max():.3e}"
    assert np.all(dT <= T_ABS), f"{what}: max |dT| {dT.max():.3e} K"
    rest = np.abs(gpu[:, ns + 1:] - ref[:, ns + 1:]) / np.maximum(np.abs(ref[:, ns + 1:]), 1e-300)
    assert np.all(rest <= 1e-10), f"{what}: conservative components {rest.max():.3e}"


@pytest.mark.parametrize("method", ["rok4e", "rkdp"])
def test_integration_replay_parity(rk, method):
    from oracle import conservative, explicit, rok4e

    w, mech, aux, U, S = _cells("small", 24, seed=6)
    m = rk.mech_load(mech)
    n = U.shape[0]
    Y = _t(U)
    st = torch.zeros(n, 4, dtype=torch.int32, device="cuda")
    tr = torch.zeros(n, 4096, dtype=torch.float64, device="cuda")
    o = rk.Opts(reactor=2, trace=tr)
    if method == "rok4e":
        rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, 4, src=_t(S), opts=o, stats=st)
    else:
        rk.rkdp_integrate(m, Y, w.dt, w.rtol, w.atol, src=_t(S), opts=o, stats=st)
    torch.cuda.synchronize()
    out, s, trace = Y.cpu().numpy(), st.cpu().numpy(), tr.cpu().numpy()
    assert np.all(s[:, 3] == 0)
    ref = np.empty_like(U)
    for c in range(n):
        rp = [(abs(h), h > 0) for h in trace[c] if h != 0.0]
        if method == "rok4e":
            f, jv_at = conservative.reactor(aux, S[c])
            ref[c], _ = rok4e.integrate(f, jv_at, U[c], w.dt, w.rtol, w.atol, 4, replay=rp)
        else:
            ref[c], _ = explicit.integrate(lambda u, s=S[c]: aux.rhs(u, s), U[c], w.dt, w.rtol, w.atol, replay=rp)
    _close(out, ref, mech.n_species, method)


def test_steady_state_is_bit_exact(rk):
    w, mech, aux, U, _ = _cells("flame1d", 16, seed=7, with_src=False)
    m = rk.mech_load(mech)
    ns = mech.n_species
    Ug = _t(U)
    S = -rk.chem_rhs_aux(m, Ug)
    S[:, ns:] = 0.0  # balancing constants cancel the species source; none on rho, rho v, rho E
    Y = Ug.clone()
    st = torch.zeros(U.shape[0], 4, dtype=torch.int32, device="cuda")
    rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, 4, src=S, opts=rk.Opts(reactor=2), stats=st)
    torch.cuda.synchronize()
    assert torch.equal(Y, Ug)
    assert np.all(st.cpu().numpy()[:, 0] == 1)


def test_unsupported_combinations_raise(rk):
    w, mech, aux, U, S = _cells("small", 4)
    m = rk.mech_load(mech)
    with pytest.raises(rk.RokError):
        rk.rok4e_integrate(m, _t(U), w.dt, w.rtol, w.atol, 4, opts=rk.Opts(reactor=2, precision=1))
