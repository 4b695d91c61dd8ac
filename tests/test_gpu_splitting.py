"""GPU splitting schemes (Sec. 3) on the 1-D reaction-diffusion system.

* Each scheme against the oracle's split step on the same grid, both
  integrating the reaction sub-steps at tight tolerance (free running).
* Scheme 0 of rk_split_step is bitwise rk_simpler_split_step.
* Second-order convergence in the split step size of the balanced schemes
  (the paper's 1-D flame shows 2nd order in T), measured on the GPU.
"""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

P = 101325.0
D = 1e-4


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1712_00953_gb300 as rk

    return rk


@pytest.fixture(scope="module")
def case():
    from synth.fields import WORKLOADS, field_tanh_front, mechanism_for

    w = WORKLOADS["flame1d"]
    mech = mechanism_for(w)
    return w, mech


@pytest.mark.parametrize("scheme", ["simpler", "strang", "simple_balanced", "simple_balanced_transport_first"])
def test_scheme_matches_oracle(rk, case, scheme):
    from oracle import splitting as osp
    from oracle.kinetics import Kinetics
    from synth.fields import field_tanh_front

    w, mech = case
    npts = 24
    _, U0 = field_tanh_front(npts, mech.n_species, w.field_seed)
    dx = 1e-2 / npts
    rtol, atol, dt = 1e-9, 1e-13, 5e-8
    m = rk.mech_load(mech)
    U = torch.tensor(U0, device="cuda")
    hc = torch.zeros(npts, dtype=torch.float64, device="cuda")
    Uo = U0.copy()
    ho = np.zeros(npts)
    kin = Kinetics(mech)
    for _ in range(2):
        rk.split_step(m, U, dt, D, dx, rtol, atol, 4, scheme, h_cell=hc)
        Uo = osp.split_step_1d(kin, Uo, P, dt, D, dx, rtol, atol, 4, scheme, h_cell=ho)
    torch.cuda.synchronize()
    g = U.cpu().numpy()
    ns = mech.n_species
    dY = np.abs(g[:, :ns] - Uo[:, :ns])
    assert np.all(dY <= 1e-8 + 1e-6 * np.abs(Uo[:, :ns])), dY.max()
    assert np.max(np.abs(g[:, ns] - Uo[:, ns])) <= 1e-6


def test_scheme_zero_is_the_simpler_entry_point(rk, case):
    from synth.fields import field_tanh_front

    w, mech = case
    _, U0 = field_tanh_front(128, mech.n_species, w.field_seed)
    m = rk.mech_load(mech)
    a = torch.tensor(U0, device="cuda")
    b = torch.tensor(U0, device="cuda")
    ha = torch.zeros(128, dtype=torch.float64, device="cuda")
    hb = torch.zeros(128, dtype=torch.float64, device="cuda")
    for _ in range(3):
        rk.simpler_split_step(m, a, w.dt, D, 1e-2 / 128, w.rtol, w.atol, 4, h_cell=ha)
        rk.split_step(m, b, w.dt, D, 1e-2 / 128, w.rtol, w.atol, 4, "simpler", h_cell=hb)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(ha, hb)


@pytest.mark.parametrize("scheme", ["simpler", "simple_balanced", "strang"])
def test_second_order_in_split_step(rk, case, scheme):
    from synth.fields import field_tanh_front

    w, mech = case
    npts = 128
    _, U0 = field_tanh_front(npts, mech.n_species, w.field_seed)
    dx = 1e-2 / npts
    m = rk.mech_load(mech)
    t_end = 4e-7

    def run(nsteps):
        U = torch.tensor(U0, device="cuda")
        hc = torch.zeros(npts, dtype=torch.float64, device="cuda")
        for _ in range(nsteps):
            rk.split_step(m, U, t_end / nsteps, D, dx, 1e-10, 1e-14, 4, scheme, h_cell=hc)
        torch.cuda.synchronize()
        return U.cpu().numpy()

    ref = run(64)
    errs = [np.max(np.abs(run(n)[:, -1] - ref[:, -1])) for n in (4, 8, 16)]
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    print(f"{scheme}: T errors {errs}, observed orders {slopes}")
    assert np.all(slopes > 1.6), (errs, slopes)


def test_transport_first_simple_balancing_is_unstable_at_large_steps(rk, case):
    """Sec. 3.3: simple balancing with the non-stiff part first is stable only
    for |B| h < 5.99; at a split step far beyond that its error dwarfs the
    Simpler scheme's, and it recovers as the step shrinks."""
    from synth.fields import field_tanh_front

    w, mech = case
    npts = 128
    _, U0 = field_tanh_front(npts, mech.n_species, w.field_seed)
    dx = 1e-2 / npts
    m = rk.mech_load(mech)
    t_end = 4e-7

    def run(scheme, nsteps):
        U = torch.tensor(U0, device="cuda")
        hc = torch.zeros(npts, dtype=torch.float64, device="cuda")
        for _ in range(nsteps):
            rk.split_step(m, U, t_end / nsteps, D, dx, 1e-10, 1e-14, 4, scheme, h_cell=hc)
        torch.cuda.synchronize()
        return U.cpu().numpy()[:, -1]

    ref = run("simpler", 64)
    e_tf = np.max(np.abs(run("simple_balanced_transport_first", 4) - ref))
    e_s = np.max(np.abs(run("simpler", 4) - ref))
    e_tf_fine = np.max(np.abs(run("simple_balanced_transport_first", 16) - ref))
    print(f"coarse step: transport-first simple balanced {e_tf:.3e} K vs Simpler {e_s:.3e} K; finer {e_tf_fine:.3e} K")
    assert e_tf > 100 * e_s
    assert e_tf_fine < 0.01 * e_tf
