"""GPU parity of the explicit Dormand-Prince 5(4) integrator (the efficiency
study's explicit reference, Sec. 4.4) against the FP64 oracle
(oracle/explicit.py): replay of the GPU's own step sequence, free-running
step counts, fixed steps, the first-same-as-last RHS count, an exact steady
state and argument errors."""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

P = 101325.0
Y_ABS, Y_REL, T_ABS = 1e-8, 1e-6, 1e-6


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1712_00953_gb300 as rk

    return rk


def _mech(name):
    from synth.fields import WORKLOADS, mechanism_for

    return WORKLOADS[name], mechanism_for(WORKLOADS[name])


def _run(rk, mech, U, dt, rtol, atol, cap=4096, opts=None, src=None):
    m = rk.mech_load(mech)
    Y = torch.tensor(U, device="cuda")
    n = U.shape[0]
    st = torch.zeros(n, 4, dtype=torch.int32, device="cuda")
    tr = torch.zeros(n, cap, dtype=torch.float64, device="cuda")
    o = opts or rk.Opts()
    o.trace = tr
    rk.rkdp_integrate(m, Y, dt, rtol, atol, opts=o, stats=st,
                      src=None if src is None else torch.tensor(src, device="cuda"))
    torch.cuda.synchronize()
    return Y.cpu().numpy(), st.cpu().numpy(), tr.cpu().numpy()


def _close(gpu, ref, ns, what):
    dY = np.abs(gpu[:, :ns] - ref[:, :ns])
    excess = dY - (Y_ABS + Y_REL * np.abs(ref[:, :ns]))
    dT = np.abs(gpu[:, ns] - ref[:, ns])
    assert np.all(excess <= 0.0), f"{what}: max Y excess {excess.max():.3e}"
    assert np.all(dT <= T_ABS), f"{what}: max |dT| {dT.max():.3e} K"


@pytest.mark.parametrize("name", ["small", "flame1d"])
def test_replay_parity_and_rhs_count(rk, name):
    from oracle import explicit
    from oracle.kinetics import Kinetics
    from synth.fields import initial_state

    w, mech = _mech(name)
    U = initial_state(w)[::16][:48]
    out, st, tr = _run(rk, mech, U, w.dt, w.rtol, w.atol)
    assert np.all(st[:, 3] == 0)
    att = st[:, 0] + st[:, 1]
    assert np.all(att <= tr.shape[1])
    assert np.all(st[:, 2] == 1 + 6 * att)  # first same as last
    replay = [[(abs(h), h > 0) for h in r if h != 0.0] for r in tr]
    ref, _ = explicit.integrate_cells(Kinetics(mech), U, P, w.dt, w.rtol, w.atol, replay=replay)
    _close(out, ref, mech.n_species, f"{name} replay")
    # free-running oracle on a few cells: same accepted/rejected counts
    ref2, infos = explicit.integrate_cells(Kinetics(mech), U[:8], P, w.dt, w.rtol, w.atol)
    same = [i for i, inf in enumerate(infos) if inf["n_accept"] == st[i, 0] and inf["n_reject"] == st[i, 1]]
    assert len(same) >= 7
    _close(out[:8][same], ref2[same], mech.n_species, f"{name} free")


def test_fixed_steps_match_oracle(rk):
    from oracle import explicit
    from oracle.kinetics import Kinetics
    from synth.fields import initial_state

    w, mech = _mech("small")
    U = initial_state(w)[:32]
    out, st, _ = _run(rk, mech, U, 1e-7, w.rtol, w.atol, opts=rk.Opts(fixed_h=1e-8))
    assert np.all(st[:, 0] == 10) and np.all(st[:, 1] == 0)
    ref, _ = explicit.integrate_cells(Kinetics(mech), U, P, 1e-7, w.rtol, w.atol, fixed_h=1e-8)
    _close(out, ref, mech.n_species, "fixed")


def test_steady_state_is_bit_exact(rk):
    from synth.fields import initial_state

    w, mech = _mech("flame1d")
    U = initial_state(w)[::64]
    m = rk.mech_load(mech)
    Ug = torch.tensor(U, device="cuda")
    src = -rk.chem_rhs(m, Ug, P)
    Y = Ug.clone()
    st = torch.zeros(U.shape[0], 4, dtype=torch.int32, device="cuda")
    rk.rkdp_integrate(m, Y, w.dt, w.rtol, w.atol, src=src, stats=st)
    torch.cuda.synchronize()
    assert torch.equal(Y, Ug)
    s = st.cpu().numpy()
    assert np.all(s[:, 0] == 1) and np.all(s[:, 1] == 0)


def test_argument_errors(rk):
    w, mech = _mech("small")
    m = rk.mech_load(mech)
    Y = torch.zeros(4, mech.n_species + 1, dtype=torch.float64, device="cuda") + 1000.0
    with pytest.raises(rk.RokError):
        rk.rkdp_integrate(m, Y, w.dt, w.rtol, w.atol, opts=rk.Opts(precision=1))
    with pytest.raises(rk.RokError):
        rk.rkdp_integrate(m, Y, -1.0, w.rtol, w.atol)
