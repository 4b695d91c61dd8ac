"""GPU splitting schemes (Sec. 3) on the 1-D reaction-diffusion system.

* Each scheme against the oracle's split step on the same grid, both
  integrating the reaction sub-steps at tight tolerance (free running).
* Scheme 0 of rk_split_step is bitwise rk_simpler_split_step.
* The domain split into slices with one ghost row per side (the multi-GPU
  layout), emulated by two slices on one GPU whose halos are copied between
  the phases, is bitwise the whole-domain split step.
* Second-order convergence in the split step size of the balanced schemes
  (the paper's 1-D flame shows 2nd order in T), measured on the GPU.
* The split step with the caller's own transport operator
  (rk_simpler_split_step_ext): bitwise the built-in step when the operator is
  the library's diffusion; with an upwind advection operator, against the
  oracle's Simpler step (Eq. simpler_balanced) with the same operator,
  replaying the GPU's reaction step sequences; without an operator, the
  reaction step alone; a failing operator stops the step with an error.
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


def test_sharded_slices_equal_whole_domain_bitwise(rk, case):
    """Two slices of a 301-point front (150 + 151 points) held with ghost
    rows, their halos copied between them before each of the four transport
    evaluations (host-ordered copies on one stream: no kernel waits on
    another), three split steps: states, carried steps and statistics equal
    rk_simpler_split_step on the whole domain bit for bit; so does the
    one-rank rk.simpler_split_step_sharded."""
    from synth.fields import field_tanh_front

    w, mech = case
    m = rk.mech_load(mech)
    npts = 301
    _, U0 = field_tanh_front(npts, mech.n_species, w.field_seed)
    dx = 1e-2 / npts
    U = torch.tensor(U0, device="cuda")
    hc = torch.zeros(npts, dtype=torch.float64, device="cuda")
    st = torch.zeros(npts, 4, dtype=torch.int32, device="cuda")
    cuts = [(0, 150), (150, npts)]
    ext = [torch.zeros(b - a + 2, U0.shape[1], dtype=torch.float64, device="cuda") for a, b in cuts]
    hs = [torch.zeros(b - a, dtype=torch.float64, device="cuda") for a, b in cuts]
    ss = [torch.zeros(b - a, 4, dtype=torch.int32, device="cuda") for a, b in cuts]
    for e, (a, b) in zip(ext, cuts):
        e[1:-1] = U[a:b]
    one = torch.zeros(npts + 2, U0.shape[1], dtype=torch.float64, device="cuda")
    one[1:-1] = U
    h1 = torch.zeros(npts, dtype=torch.float64, device="cuda")
    for step in range(3):
        rk.simpler_split_step(m, U, w.dt, D, dx, w.rtol, w.atol, 4, h_cell=hc, stats=st)
        rk.simpler_split_step_sharded(m, one, w.dt, D, dx, w.rtol, w.atol, 4, h_cell=h1)

        def react(r):
            return lambda Ur, Tn: rk.rok4e_integrate(m, Ur, w.dt, w.rtol, w.atol, 4, src=Tn, h_cell=hs[r],
                                                     stats=ss[r])

        gens = [rk.simpler_split_step_phases(react(r), rk.GhostTransport(), ext[r], w.dt, D, dx) for r in (0, 1)]
        while True:
            xs = [next(g, None) for g in gens]
            if all(x is None for x in xs):
                break
            assert all(x is not None for x in xs)
            n0, n1 = xs[0].shape[0] - 2, xs[1].shape[0] - 2
            xs[0][0] = xs[0][1]  # the domain's ends: zero gradient
            xs[1][n1 + 1] = xs[1][n1]
            xs[0][n0 + 1] = xs[1][1]  # the halo between the slices
            xs[1][0] = xs[0][n0]
        torch.cuda.synchronize()
        got = torch.cat([e[1:-1] for e in ext])
        assert torch.equal(got, U), step
        assert torch.equal(torch.cat(hs), hc), step
        assert torch.equal(torch.cat(ss), st), step
        assert torch.equal(one[1:-1], U), step
        assert torch.equal(h1, hc), step


def _upwind_torch(a, dx):
    def T(X, TX):  # first-order upwind advection at speed a > 0; the inflow point keeps its state
        TX[0].zero_()
        torch.mul(X[1:] - X[:-1], -a / dx, out=TX[1:])
    return T


def _upwind_numpy(U, a, dx):
    TU = np.zeros_like(U)
    TU[1:] = (U[1:] - U[:-1]) * (-a / dx)
    return TU


def test_split_step_ext_with_builtin_diffusion_is_bitwise(rk, case):
    from synth.fields import field_tanh_front

    w, mech = case
    npts = 256
    _, U0 = field_tanh_front(npts, mech.n_species, w.field_seed)
    dx = 1e-2 / npts
    m = rk.mech_load(mech)
    res = []
    for ext in (False, True):
        U = torch.tensor(U0, device="cuda")
        hc = torch.zeros(npts, dtype=torch.float64, device="cuda")
        st = torch.zeros(npts, 4, dtype=torch.int32, device="cuda")
        for _ in range(3):
            if ext:
                rk.simpler_split_step_ext(m, U, w.dt, w.rtol, w.atol, 4, h_cell=hc, stats=st,
                                          transport=lambda X, TX: rk.diffusion_1d(X, D, dx, out=TX))
            else:
                rk.simpler_split_step(m, U, w.dt, D, dx, w.rtol, w.atol, 4, h_cell=hc, stats=st)
        torch.cuda.synchronize()
        res.append((U.cpu(), hc.cpu(), st.cpu()))
    for a, b in zip(res[0], res[1]):
        assert torch.equal(a, b)


def test_split_step_ext_upwind_advection_vs_oracle(rk, case):
    from oracle import rok4e as orok
    from oracle import splitting as osp
    from oracle.kinetics import Kinetics
    from synth.fields import field_tanh_front

    w, mech = case
    kin = Kinetics(mech)
    npts, a = 48, 10.0
    _, U0 = field_tanh_front(npts, mech.n_species, w.field_seed)
    dx = 1e-2 / npts
    m = rk.mech_load(mech)
    U = torch.tensor(U0, device="cuda")
    hc = torch.zeros(npts, dtype=torch.float64, device="cuda")
    trace = torch.zeros(npts, 4096, dtype=torch.float64, device="cuda")
    Uo, h_or = U0.copy(), np.zeros(npts)
    ns = mech.n_species
    for step in range(2):
        trace.zero_()
        rk.simpler_split_step_ext(m, U, w.dt, w.rtol, w.atol, 4, h_cell=hc, opts=rk.Opts(trace=trace),
                                  transport=_upwind_torch(a, dx))
        torch.cuda.synchronize()
        tr = trace.cpu().numpy()
        # the oracle's Simpler step with the same operator, reaction sub-steps replayed
        Tn = _upwind_numpy(Uo, a, dx)
        U1 = Uo.copy()
        for c in range(npts):
            f, jv_at = orok.reactor(kin, P, Tn[c], "analytic")
            U1[c], inf = orok.integrate(f, jv_at, Uo[c], w.dt, w.rtol, w.atol, 4, h0=h_or[c] if step else None,
                                        replay=[(abs(h), h > 0) for h in tr[c] if h != 0.0])
            h_or[c] = inf["h_last"]
        Uo = osp.ssprk3(U1, w.dt / 2, lambda V: _upwind_numpy(V, a, dx) - Tn)
        got = U.cpu().numpy()
        dY = np.abs(got[:, :ns] - Uo[:, :ns])
        dT = np.abs(got[:, ns] - Uo[:, ns])
        print(f"upwind transport, split step {step}: max |dY| {dY.max():.3e}, max |dT| {dT.max():.3e} K")
        assert np.all(dY <= 1e-8 + 1e-6 * np.abs(Uo[:, :ns]))
        assert dT.max() <= 1e-6
    # the transport moved the front: the state differs from a pure reaction step
    Ur = torch.tensor(U0, device="cuda")
    for _ in range(2):
        rk.simpler_split_step_ext(m, Ur, w.dt, w.rtol, w.atol, 4)
    torch.cuda.synchronize()
    assert float((Ur - U).abs()[:, ns].max()) > 1e-3


def test_split_step_ext_without_transport_is_the_reaction_step(rk, case):
    from synth.fields import field_tanh_front

    w, mech = case
    npts = 128
    _, U0 = field_tanh_front(npts, mech.n_species, w.field_seed)
    m = rk.mech_load(mech)
    U1, U2 = torch.tensor(U0, device="cuda"), torch.tensor(U0, device="cuda")
    rk.simpler_split_step_ext(m, U1, w.dt, w.rtol, w.atol, 4)
    rk.rok4e_integrate(m, U2, w.dt, w.rtol, w.atol, 4)
    torch.cuda.synchronize()
    assert torch.equal(U1, U2)


def test_split_step_ext_failing_transport_stops_the_step(rk, case):
    from synth.fields import field_tanh_front

    w, mech = case
    _, U0 = field_tanh_front(32, mech.n_species, w.field_seed)
    m = rk.mech_load(mech)
    U = torch.tensor(U0, device="cuda")

    def bad(X, TX):
        raise ValueError("transport not available")

    with pytest.raises(ValueError, match="transport not available"):
        rk.simpler_split_step_ext(m, U, w.dt, w.rtol, w.atol, 4, transport=bad)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(U.cpu().numpy(), U0)  # it failed before the reaction sub-step
