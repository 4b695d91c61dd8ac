"""GPU checks of the fixed-step integration and its discrete adjoint.

* rk_rok4e_fixed_steps against the oracle's fixed-step integration.
* The adjoint's d T_final / d ln A_j and d T_final / d u0 against the oracle's
  complex-step derivatives of the same fixed-step computation (exact to
  rounding), on a sample of parameters, and against GPU central differences.
* The torch.autograd.Function wrapper returns the adjoint's gradient.
"""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

P = 101325.0


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1712_00953_gb300 as rk

    return rk


def _setup(name, ncell):
    from synth.fields import WORKLOADS, field_uniform, mechanism_for

    w = WORKLOADS[name]
    mech = mechanism_for(w)
    U = field_uniform(ncell, mech.n_species, w.field_seed, 1000.0, 1500.0)
    return w, mech, U


def _adjoint_T(rk, mech, U, h, nsteps, M=4):
    m = rk.mech_load(mech)
    Y = torch.tensor(U, device="cuda")
    n = U.shape[0]
    ck = torch.empty(nsteps + 1, n, U.shape[1], dtype=torch.float64, device="cuda")
    rk.rok4e_fixed_steps(m, Y, h, nsteps, M, checkpoints=ck)
    ubar = torch.zeros_like(Y)
    ubar[:, -1] = 1.0
    g0 = torch.empty_like(Y)
    grad, g0 = rk.rok4e_adjoint(m, ck, ubar, h, nsteps, M, grad_u0=g0)
    torch.cuda.synchronize()
    return Y.cpu().numpy(), ck.cpu().numpy(), grad.cpu().numpy(), g0.cpu().numpy()


def test_fixed_steps_match_oracle(rk):
    from oracle import rok4e as orok
    from oracle.kinetics import Kinetics

    w, mech, U = _setup("small", 6)
    h, nsteps = 2e-8, 10
    Y, ck, _, _ = _adjoint_T(rk, mech, U, h, nsteps)
    ref, _ = orok.integrate_cells(Kinetics(mech), U, P, h * nsteps, 1.0, 1.0, 4, fixed_h=h)
    ns = mech.n_species
    assert np.all(np.abs(Y[:, :ns] - ref[:, :ns]) <= 1e-8 + 1e-6 * np.abs(ref[:, :ns]))
    assert np.max(np.abs(Y[:, ns] - ref[:, ns])) <= 1e-6
    np.testing.assert_array_equal(ck[0], U)
    np.testing.assert_array_equal(ck[-1], Y)


@pytest.mark.parametrize("name,nsteps,h", [("small", 10, 2e-8), ("mixed", 8, 1e-8)])
def test_adjoint_matches_oracle_complex_step(rk, name, nsteps, h):
    from oracle import adjoint as oad
    from oracle.kinetics import Kinetics

    w, mech, U = _setup(name, 3)
    Y, ck, grad, g0 = _adjoint_T(rk, mech, U, h, nsteps)
    kin = Kinetics(mech)
    js = np.argsort(-np.abs(grad))[:6]  # the largest sensitivities plus two random ones
    js = np.concatenate([js, np.random.default_rng(0).choice(mech.n_reactions, 2, replace=False)])
    ref = sum(oad.grad_complex_step(kin, U[c], P, h, nsteps, 4, js) for c in range(U.shape[0]))
    scale = np.max(np.abs(grad))
    print(f"{name}: adjoint vs complex step, max |diff| / max |grad| = {np.max(np.abs(grad[js] - ref)) / scale:.3e}")
    assert np.max(np.abs(grad[js] - ref)) <= 1e-7 * scale
    # d T_final / d u0 for one cell, all components, by complex step on the state
    c = 0
    N = U.shape[1]
    cs = np.empty(N)
    for e in range(N):
        u = U[c].astype(complex)
        u[e] += 1e-30j
        cs[e] = np.imag(oad.final_state(kin, u, P, h, nsteps, 4)[-1]) / 1e-30
    assert np.max(np.abs(g0[c] - cs)) <= 1e-7 * np.max(np.abs(cs))


def test_adjoint_matches_gpu_central_differences(rk):
    w, mech, U = _setup("mixed", 64)
    h, nsteps = 1e-8, 8
    Y, ck, grad, _ = _adjoint_T(rk, mech, U, h, nsteps)
    order = np.argsort(-np.abs(grad))[:12]
    d = 1e-4
    fd = []
    for j in order:
        vals = []
        for sgn in (1.0, -1.0):
            mk = mech.copy()
            mk.arrh[j, 0] *= np.exp(sgn * d)
            m = rk.mech_load(mk)
            Yj = torch.tensor(U, device="cuda")
            rk.rok4e_fixed_steps(m, Yj, h, nsteps, 4)
            vals.append(Yj[:, -1].sum().item())
        fd.append((vals[0] - vals[1]) / (2 * d))
    fd = np.array(fd)
    rel = np.abs(grad[order] - fd) / np.abs(grad[order])
    print(f"adjoint vs central differences (d = {d}): max relative difference {rel.max():.2e}")
    assert rel.max() < 1e-5


@pytest.mark.parametrize("name", ["small", "mixed", "adjoint"])
def test_adjoint_lane_counts_agree(rk, name):
    """4, 8, 16 and 32 lanes per cell split the same loops differently, so the
    gradients agree to rounding; a repeated call with the same lane count
    gives the same bits (every sum has a fixed order)."""
    w, mech, U = _setup(name, 40)
    h, nsteps = 1e-8, 4
    m = rk.mech_load(mech)
    Y = torch.tensor(U, device="cuda")
    ck = torch.empty(nsteps + 1, U.shape[0], U.shape[1], dtype=torch.float64, device="cuda")
    rk.rok4e_fixed_steps(m, Y, h, nsteps, 4, checkpoints=ck)
    ubar = torch.zeros_like(Y)
    ubar[:, -1] = 1.0
    res = {}
    for G in (4, 8, 16, 32, 8):
        g0 = torch.empty_like(Y)
        grad, g0 = rk.rok4e_adjoint(m, ck, ubar, h, nsteps, 4, grad_u0=g0, lanes_per_cell=G)
        torch.cuda.synchronize()
        if G in res:
            assert torch.equal(grad, res[G][0]) and torch.equal(g0, res[G][1])
        res[G] = (grad.clone(), g0.clone())
    for G in (4, 16, 32):
        for a, b in zip(res[G], res[8]):
            assert torch.max(torch.abs(a - b)) <= 1e-12 * torch.max(torch.abs(b)), (G, float(torch.max(torch.abs(a - b))))
    with pytest.raises(rk.RokError, match="lanes_per_cell"):
        rk.rok4e_adjoint(m, ck, ubar, h, nsteps, 4, lanes_per_cell=12)


def test_autograd_function(rk):
    from paper_1712_00953_gb300 import FixedStepROK4E

    w, mech, U = _setup("small", 16)
    lnA = torch.tensor(np.log(mech.arrh[:, 0]), dtype=torch.float64, requires_grad=True)
    Y0 = torch.tensor(U, device="cuda", requires_grad=True)
    Y = FixedStepROK4E.apply(lnA, Y0, mech, 2e-8, 10, 4)
    loss = Y[:, -1].sum()
    loss.backward()
    _, _, grad, g0 = _adjoint_T(rk, mech, U, 2e-8, 10)
    np.testing.assert_allclose(lnA.grad.numpy(), grad, rtol=0, atol=1e-12 * np.abs(grad).max())
    np.testing.assert_allclose(Y0.grad.cpu().numpy(), g0, rtol=0, atol=1e-12 * np.abs(g0).max())


def test_adjoint_full_size_sampled(rk):
    """The adjoint workload at full size (4096 cells, 100 species / 500
    reactions, 50 fixed steps of 1e-7 s): the adjoint seeded on two sampled
    cells' final temperatures (the coldest and the hottest), checked along a
    random direction in ln A against the oracle's complex-step directional
    derivative of those two cells.  The hot cell's derivative is ill-conditioned
    (a 1e-13 relative change of its initial temperature moves it by ~1e-6
    relative in the oracle itself), so the bar per cell is ten times the
    oracle's own spread under such perturbations, plus 1e-9 relative."""
    from oracle import adjoint as oad
    from oracle.kinetics import Kinetics
    from synth.fields import WORKLOADS, initial_state, mechanism_for

    w = WORKLOADS["adjoint"]
    mech = mechanism_for(w)
    U = initial_state(w)
    n, N = U.shape
    nsteps, h = w.n_steps, w.dt
    m = rk.mech_load(mech)
    Y = torch.tensor(U, device="cuda")
    ck = torch.empty(nsteps + 1, n, N, dtype=torch.float64, device="cuda")
    rk.rok4e_fixed_steps(m, Y, h, nsteps, w.krylov_dim, checkpoints=ck)
    order = np.argsort(U[:, -1])
    cells = [int(order[0]), int(order[-1])]  # coldest and hottest
    ubar = torch.zeros_like(Y)
    ubar[cells, -1] = 1.0
    grad, _ = rk.rok4e_adjoint(m, ck, ubar, h, nsteps, w.krylov_dim)
    torch.cuda.synchronize()
    grad = grad.cpu().numpy()
    assert np.all(np.isfinite(grad))
    kin = Kinetics(mech)
    d = np.random.default_rng(7).normal(size=mech.n_reactions)
    d /= np.linalg.norm(d)
    lnA = kin.lnA_input.astype(complex) + 1j * oad.CS_EPS * d
    ref, tol = 0.0, 0.0
    for c in cells:
        vals = []
        for pert in (0.0, 1e-13, -1e-13):
            u0 = U[c].copy()
            u0[-1] *= 1.0 + pert
            uf = oad.final_state(kin, u0.astype(complex), P, h, nsteps, w.krylov_dim, lnA)
            vals.append(float(np.imag(uf[-1])) / oad.CS_EPS)
        ref += vals[0]
        tol += 10.0 * max(abs(vals[1] - vals[0]), abs(vals[2] - vals[0])) + 1e-9 * abs(vals[0])
    got = float(grad @ d)
    print(f"full-size adjoint, directional derivative: GPU {got:.10e}, oracle {ref:.10e}, bar {tol:.2e}")
    assert abs(got - ref) <= tol
