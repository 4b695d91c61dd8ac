"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances.  The chemistry source and its Jacobian-vector product are the same
FP64 arithmetic on both sides up to summation order and contraction, so they
agree to ~1e-12 of the row scale.  Integrated states are compared with the
bar the library is built to: |dY| <= 1e-8 + 1e-6 |Y| and |dT| <= 1e-6 K.
"Replay" runs the oracle on the GPU's recorded step sequence (same h, same
accept/reject decisions), which removes decisions that flip when an error
estimate sits at 1 to within rounding.
"""

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


def _assert_state_close(gpu, ref, ns, what=""):
    dY = np.abs(gpu[:, :ns] - ref[:, :ns])
    excess = dY - (Y_ABS + Y_REL * np.abs(ref[:, :ns]))
    dT = np.abs(gpu[:, ns] - ref[:, ns])
    assert np.all(excess <= 0.0), f"{what}: max Y excess {excess.max():.3e} (max |dY| {dY.max():.3e})"
    assert np.all(dT <= T_ABS), f"{what}: max |dT| {dT.max():.3e} K"
    return dY.max(), dT.max()


def _replay_of(trace_row):
    return [(abs(h), h > 0) for h in trace_row if h != 0.0]


@pytest.mark.parametrize("name", ["small", "flame1d", "batched", "adjoint"])
def test_chem_rhs_matches_oracle(rk, name):
    from oracle.kinetics import Kinetics
    from synth.fields import field_uniform, initial_state

    w, mech = _mech(name)
    kin = Kinetics(mech)
    if name == "batched" or name == "adjoint":
        U = field_uniform(67, mech.n_species, 7, 300.0, 3000.0)
    else:
        U = initial_state(w)[::7][:67]
    src = np.random.default_rng(3).normal(size=U.shape) * 10.0
    m = rk.mech_load(mech)
    Ug = torch.tensor(U, device="cuda")
    for s in (None, src):
        out = rk.chem_rhs(m, Ug, P, src=None if s is None else torch.tensor(s, device="cuda")).cpu().numpy()
        ref = np.array([kin.rhs(u, P, None if s is None else s[i]) for i, u in enumerate(U)])
        scale = np.max(np.abs(ref), axis=1, keepdims=True)
        assert np.max(np.abs(out - ref) / scale) < 1e-11


@pytest.mark.parametrize("name", ["small", "flame1d", "batched"])
def test_chem_jvp_matches_oracle(rk, name):
    from oracle.kinetics import Kinetics
    from synth.fields import field_uniform

    w, mech = _mech(name)
    kin = Kinetics(mech)
    U = field_uniform(40, mech.n_species, 11, 500.0, 2800.0)
    V = np.random.default_rng(5).normal(size=U.shape)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    m = rk.mech_load(mech)
    Ug, Vg = torch.tensor(U, device="cuda"), torch.tensor(V, device="cuda")
    out = rk.chem_jvp(m, Ug, Vg, P, mode=0).cpu().numpy()
    ref = np.array([kin.jvp(u, P, v) for u, v in zip(U, V)])
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.max(np.abs(out - ref) / scale) < 1e-10
    fd = rk.chem_jvp(m, Ug, Vg, P, mode=1).cpu().numpy()
    ref_fd = np.array([kin.jvp_fd(u, P, v) for u, v in zip(U, V)])
    assert np.max(np.abs(fd - ref_fd) / scale) < 1e-5


def _integrate(rk, mech, U, w, M=4, src=None, h_cell=None, opts=None, cap=8192):
    m = rk.mech_load(mech)
    Y = torch.tensor(U, device="cuda")
    n = U.shape[0]
    stats = torch.zeros(n, 4, dtype=torch.int32, device="cuda")
    trace = torch.zeros(n, cap, dtype=torch.float64, device="cuda")
    o = opts or rk.Opts()
    o.trace = trace
    rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, M, src=None if src is None else torch.tensor(src, device="cuda"),
                       h_cell=h_cell, opts=o, stats=stats)
    torch.cuda.synchronize()
    return Y.cpu().numpy(), stats.cpu().numpy(), trace.cpu().numpy()


def test_small_workload_replay_and_free_parity(rk):
    from oracle import rok4e as orok
    from oracle.kinetics import Kinetics
    from synth.fields import initial_state

    w, mech = _mech("small")
    kin = Kinetics(mech)
    U = initial_state(w)
    out, st, tr = _integrate(rk, mech, U, w)
    assert np.all(st[:, 3] == 0)
    assert np.all(st[:, 0] + st[:, 1] <= tr.shape[1])
    sel = np.arange(0, U.shape[0], 4)  # 64 of the 256 cells through the oracle
    ref, infos = orok.integrate_cells(kin, U[sel], P, w.dt, w.rtol, w.atol, 4,
                                      replay=[_replay_of(tr[i]) for i in sel])
    _assert_state_close(out[sel], ref, mech.n_species, "replay")
    # free-running oracle: same decisions on (nearly) every cell
    ref2, infos2 = orok.integrate_cells(kin, U[sel[:16]], P, w.dt, w.rtol, w.atol, 4)
    same = [i for i, inf in enumerate(infos2) if inf["n_accept"] == st[sel[i], 0] and inf["n_reject"] == st[sel[i], 1]]
    assert len(same) >= 14
    _assert_state_close(out[sel[:16]][same], ref2[same], mech.n_species, "free")


def test_fd_jacobian_mode_parity(rk):
    from oracle import rok4e as orok
    from oracle.kinetics import Kinetics
    from synth.fields import initial_state

    w, mech = _mech("small")
    U = initial_state(w)[:12]
    out, st, tr = _integrate(rk, mech, U, w, opts=rk.Opts(jv_mode=1))
    ref, _ = orok.integrate_cells(Kinetics(mech), U, P, w.dt, w.rtol, w.atol, 4, jv_mode="fd",
                                  replay=[_replay_of(r) for r in tr])
    _assert_state_close(out, ref, mech.n_species, "fd replay")


@pytest.mark.parametrize("M", [1, 3, 6, 8])
def test_krylov_dimensions(rk, M):
    from oracle import rok4e as orok
    from oracle.kinetics import Kinetics
    from synth.fields import initial_state

    w, mech = _mech("small")
    U = initial_state(w)[20:26]
    out, st, tr = _integrate(rk, mech, U, w, M=M)
    ref, _ = orok.integrate_cells(Kinetics(mech), U, P, w.dt, w.rtol, w.atol, M,
                                  replay=[_replay_of(r) for r in tr])
    _assert_state_close(out, ref, mech.n_species, f"M={M}")


def test_krylov_dimension_clamped_to_state_size(rk):
    from oracle import rok4e as orok
    from oracle.kinetics import Kinetics
    from synth.mechanism import single_reaction_mechanism
    from synth.fields import WORKLOADS

    mech = single_reaction_mechanism([0, 1], [2], [(0, 1, 1, 0), (0, 1, 0, 1), (0, 2, 1, 1)], 1e12, 0.5, 3.0e4)
    w = WORKLOADS["small"]
    U = np.array([[0.3, 0.3, 0.4, 1400.0], [0.1, 0.6, 0.3, 1700.0]])
    out, st, tr = _integrate(rk, mech, U, w, M=8)
    ref, _ = orok.integrate_cells(Kinetics(mech), U, P, w.dt, w.rtol, w.atol, 8,
                                  replay=[_replay_of(r) for r in tr])
    _assert_state_close(out, ref, 3, "N=4, M=8")


@pytest.mark.parametrize("lanes", [8, 16])
def test_lanes_per_cell_variants_agree(rk, lanes):
    from synth.fields import initial_state

    w, mech = _mech("small")
    U = initial_state(w)[:64]
    a, sa, _ = _integrate(rk, mech, U, w)
    b, sb, _ = _integrate(rk, mech, U, w, opts=rk.Opts(lanes_per_cell=lanes))
    _assert_state_close(b, a, mech.n_species, f"G={lanes}")


def test_queue_orders_are_bitwise_identical(rk):
    """Every cell's arithmetic is independent of which warp, block or SM runs
    it: the interleaved, longest-first and static-bin queues (with several
    block shapes) give bitwise identical states and carried steps."""
    from synth.fields import initial_state

    w, mech = _mech("flame1d")
    U = initial_state(w)[::2]
    m = rk.mech_load(mech)
    n = U.shape[0]
    h0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    Y0 = torch.tensor(U, device="cuda")
    rk.rok4e_integrate(m, Y0, w.dt, w.rtol, w.atol, 4, h_cell=h0)  # carried steps for the cost order
    outs = []
    for order, cpb, bps in [(1, 4, 0), (2, 4, 0), (3, 4, 0), (3, 16, 1), (3, 6, 0), (3, 8, 2)]:
        Y = Y0.clone()
        hc = h0.clone()
        rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, 4, h_cell=hc,
                           opts=rk.Opts(queue_order=order, cells_per_block=cpb, blocks_per_sm=bps))
        torch.cuda.synchronize()
        outs.append((Y.cpu(), hc.cpu()))
    for Y, hc in outs[1:]:
        assert torch.equal(Y, outs[0][0]) and torch.equal(hc, outs[0][1])


def test_steady_state_is_bit_exact(rk):
    from synth.fields import initial_state

    w, mech = _mech("flame1d")
    U = initial_state(w)[::64]
    m = rk.mech_load(mech)
    Ug = torch.tensor(U, device="cuda")
    src = -rk.chem_rhs(m, Ug, P)  # balancing source: f(U) = R(U) - R(U) = 0 exactly
    Y = Ug.clone()
    stats = torch.zeros(U.shape[0], 4, dtype=torch.int32, device="cuda")
    rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, 4, src=src, stats=stats)
    torch.cuda.synchronize()
    assert torch.equal(Y, Ug)
    st = stats.cpu().numpy()
    assert np.all(st[:, 0] == 1) and np.all(st[:, 1] == 0)


def test_conservation_on_gpu(rk):
    from oracle.kinetics import element_totals
    from synth.fields import initial_state

    w, mech = _mech("small")
    U = initial_state(w)
    out, st, _ = _integrate(rk, mech, U, w, cap=1)
    ns = mech.n_species
    e0 = element_totals(mech, U[:, :ns])
    e1 = element_totals(mech, out[:, :ns])
    assert np.max(np.abs(e1 - e0)) < 1e-12 * np.abs(e0).max()
    assert np.max(np.abs(out[:, :ns].sum(1) - U[:, :ns].sum(1))) < 1e-13


def test_edge_cases(rk):
    from synth.fields import initial_state

    w, mech = _mech("small")
    m = rk.mech_load(mech)
    # empty launch is a no-op
    Y0 = torch.zeros(0, mech.n_state, dtype=torch.float64, device="cuda")
    rk.rok4e_integrate(m, Y0, w.dt, w.rtol, w.atol, 4)
    # a non-finite cell fails alone; its neighbours are unaffected
    U = initial_state(w)[:5].copy()
    U[2, 0] = np.nan
    good, _, _ = _integrate(rk, mech, np.delete(U, 2, axis=0), w, cap=1)
    out, st, _ = _integrate(rk, mech, U, w, cap=1)
    assert st[2, 3] in (2, 3)
    np.testing.assert_array_equal(np.delete(out, 2, axis=0), good)
    # attempt cap reached -> status 1, call still succeeds
    out, st, _ = _integrate(rk, mech, U[:2], w, opts=rk.Opts(max_attempts=2), cap=1)
    assert np.all(st[:, 3] == 1) and np.all(st[:, 0] + st[:, 1] == 2)
    # invalid arguments raise
    with pytest.raises(rk.RokError):
        rk.rok4e_integrate(m, torch.tensor(U, device="cuda"), -1.0, w.rtol, w.atol, 4)
    with pytest.raises(rk.RokError):
        rk.rok4e_integrate(m, torch.tensor(U, device="cuda"), w.dt, w.rtol, w.atol, 9)


def test_fixed_step_mode(rk):
    from oracle import rok4e as orok
    from oracle.kinetics import Kinetics
    from synth.fields import field_uniform

    w, mech = _mech("adjoint")
    U = field_uniform(4, mech.n_species, w.field_seed)
    h = w.dt / 10
    out, st, _ = _integrate(rk, mech, U, w, opts=rk.Opts(fixed_h=h), cap=1)
    assert np.all(st[:, 0] == 10) and np.all(st[:, 1] == 0)
    ref, _ = orok.integrate_cells(Kinetics(mech), U, P, w.dt, w.rtol, w.atol, 4, fixed_h=h)
    _assert_state_close(out, ref, mech.n_species, "fixed")


def test_batched_full_size_sampled_cells(rk):
    """The 2^20-cell workload in the benchmark's launch configuration; a
    temperature-stratified sample of cells is replayed through the oracle and
    every cell is checked for conservation and status."""
    from oracle import rok4e as orok
    from oracle.kinetics import Kinetics, element_totals
    from synth.fields import initial_state

    w, mech = _mech("batched")
    U = initial_state(w)
    n = U.shape[0]
    m = rk.mech_load(mech)
    Y = torch.tensor(U, device="cuda")
    stats = torch.zeros(n, 4, dtype=torch.int32, device="cuda")
    rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, w.krylov_dim, stats=stats)
    torch.cuda.synchronize()
    out = Y.cpu().numpy()
    st = stats.cpu().numpy()
    assert np.all(st[:, 3] == 0)
    ns = mech.n_species
    e0 = element_totals(mech, U[:, :ns])
    e1 = element_totals(mech, out[:, :ns])
    assert np.max(np.abs(e1 - e0)) < 1e-11 * np.abs(e0).max()
    order = np.argsort(U[:, ns])
    sel = order[np.linspace(0, n - 1, 12).astype(int)]
    # rerun the sample with a trace to replay it exactly
    o2, s2, tr = _integrate(rk, mech, U[sel], w, cap=4096)
    np.testing.assert_array_equal(o2, out[sel])  # same cells, same result in a smaller launch
    ref, _ = orok.integrate_cells(Kinetics(mech), U[sel], P, w.dt, w.rtol, w.atol, w.krylov_dim,
                                  replay=[_replay_of(r) for r in tr])
    _assert_state_close(o2, ref, ns, "batched sample")


def test_diffusion_operator(rk):
    from oracle import splitting as osp

    U = np.random.default_rng(1).normal(size=(97, 7))
    out = rk.diffusion_1d(torch.tensor(U, device="cuda"), 1e-4, 1e-3).cpu().numpy()
    ref = osp.diffusion_op(U, 1e-4, 1e-3)
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(ref))


def test_simpler_split_step_1d_parity(rk):
    from oracle import splitting as osp
    from oracle.kinetics import Kinetics
    from synth.fields import WORKLOADS, field_tanh_front

    w, mech = _mech("flame1d")
    kin = Kinetics(mech)
    npts = 48
    _, U = field_tanh_front(npts, mech.n_species, w.field_seed)
    dx = 1e-2 / npts
    D = 1e-4
    m = rk.mech_load(mech)
    Ug = torch.tensor(U, device="cuda")
    hc = torch.zeros(npts, dtype=torch.float64, device="cuda")
    trace = torch.zeros(npts, 4096, dtype=torch.float64, device="cuda")
    Uo = U.copy()
    h_or = np.zeros(npts)
    for step in range(2):
        trace.zero_()
        rk.simpler_split_step(m, Ug, w.dt, D, dx, w.rtol, w.atol, 4, h_cell=hc, opts=rk.Opts(trace=trace))
        torch.cuda.synchronize()
        tr = trace.cpu().numpy()
        Uo, h_or, _, _ = osp.simpler_split_step_1d(kin, Uo, P, w.dt, D, dx, w.rtol, w.atol, 4,
                                                   h_cell=h_or, replay=[_replay_of(r) for r in tr])
        _assert_state_close(Ug.cpu().numpy(), Uo, mech.n_species, f"split step {step}")


def test_flame1d_full_size_split_steps_sampled(rk):
    """The 2048-point flame1d Simpler split step at full size in the
    benchmark's launch configuration (carried h_cell, default queue order and
    block shape), two steps from the initial field.  Each step is checked at
    sampled points -- the hottest cell, the steepest temperature gradient, the
    middle and both ends -- against the oracle started from the GPU's own
    input state: the reaction sub-step of the seven points around each sample
    is replayed with the full field's T(U_n), and the one-step SSP-RK3
    transport correction, whose stencil reaches three points, then gives the
    sample exactly as over the whole field."""
    from oracle import splitting as osp
    from oracle.kinetics import Kinetics
    from synth.fields import field_tanh_front

    w, mech = _mech("flame1d")
    kin = Kinetics(mech)
    _, U0 = field_tanh_front(w.n_cells, mech.n_species, w.field_seed)
    npts = U0.shape[0]
    assert npts == 2048
    dx, D = 1e-2 / npts, 1e-4
    ns = mech.n_species
    m = rk.mech_load(mech)
    Ug = torch.tensor(U0, device="cuda")
    hc = torch.zeros(npts, dtype=torch.float64, device="cuda")
    trace = torch.zeros(npts, 1024, dtype=torch.float64, device="cuda")
    stats = torch.zeros(npts, 4, dtype=torch.int32, device="cuda")
    for step in range(2):
        Un, hn = Ug.cpu().numpy(), hc.cpu().numpy()
        trace.zero_()
        rk.simpler_split_step(m, Ug, w.dt, D, dx, w.rtol, w.atol, w.krylov_dim, h_cell=hc, stats=stats,
                              opts=rk.Opts(trace=trace))
        torch.cuda.synchronize()
        out, st, tr = Ug.cpu().numpy(), stats.cpu().numpy(), trace.cpu().numpy()
        assert np.all(st[:, 3] == 0) and np.all(np.isfinite(out))
        attempts = st[:, 0] + st[:, 1]
        assert attempts.max() <= trace.shape[1]
        picks = (int(np.argmax(attempts)), int(np.argmax(np.abs(np.diff(Un[:, ns])))), npts // 2, 0, npts - 1)
        centres = sorted({min(max(c, 3), npts - 4) for c in picks})
        cells = sorted({c + d for c in centres for d in range(-3, 4)})
        replay = [_replay_of(tr[c]) if c in cells else None for c in range(npts)]
        ref, _, _, _ = osp.simpler_split_step_1d(kin, Un, P, w.dt, D, dx, w.rtol, w.atol, w.krylov_dim,
                                                 h_cell=hn, replay=replay, cells=cells)
        _assert_state_close(out[centres], ref[centres], ns, f"full-size split step {step}")


def _ulps(a, b):
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    return np.abs(ia - ib)


def test_table_exp_matches_cuda_exp(rk):
    """The kernels' table-driven exp (Tang 1989) against CUDA's exp: within 2 ulp
    on the fast path, identical on the fallback range and special values."""
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-707.9, 707.9, 400000), rng.uniform(-3, 3, 200000),
                        rng.uniform(-1e-3, 1e-3, 50000), np.linspace(-745, 709.7, 5001),
                        [0.0, -0.0, 1e-300, -1e-300, 708.0, -708.0, 709.78, -745.2, np.inf, -np.inf, np.nan]])
    xt = torch.tensor(x, device="cuda")
    ref = torch.exp(xt).cpu().numpy()
    tiny = np.finfo(float).tiny
    for which, sign in ((0, 1.0), (1, 1.0), (2, -1.0)):
        y = rk.eval_exp(xt, which).cpu().numpy()
        r = ref if sign > 0 else torch.exp(-xt).cpu().numpy()
        normal = np.isfinite(r) & (r >= tiny)
        assert np.max(_ulps(y[normal], r[normal])) <= 2
        # NaN, infinities, zero and subnormal results come from the library path
        other = ~normal
        assert np.array_equal(np.isnan(y[other]), np.isnan(r[other]))
        keep = other & ~np.isnan(r)
        assert np.array_equal(y[keep], r[keep])


def test_mixed_exp_close_to_cuda_exp(rk):
    """The mixed-precision exp (FP64 reduction and reconstruction, FP32 for the
    polynomial's small term) within 2e-12 relative of CUDA's exp."""
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-707.9, 707.9, 400000), rng.uniform(-3, 3, 200000), [0.0, 1e-300]])
    xt = torch.tensor(x, device="cuda")
    for which, sign in ((3, 1.0), (4, 1.0), (5, -1.0)):
        y = rk.eval_exp(xt, which).cpu().numpy()
        r = torch.exp(sign * xt).cpu().numpy()
        assert np.max(np.abs(y - r) / r) < 2e-12


def test_table_log_and_newton_reciprocal_match_cuda(rk):
    """The kernels' table-driven ln (Tang 1990) against CUDA's log: within
    3 ulp or 2.5e-16 absolute (near x = 1, where the intervals below 1 cancel
    against -ln 2); the Newton reciprocal within 1 ulp of the IEEE division;
    both identical to the library on their fallback ranges (zero, negative,
    subnormal, huge, infinite, NaN)."""
    rng = np.random.default_rng(2)
    tiny = np.finfo(float).tiny
    special = [1.0, 2.0, 0.5, 1.0 - 2.0 ** -53, 1.0 + 2.0 ** -52, tiny, np.finfo(float).max, 5e-324, 0.0,
               -0.0, -1.0, np.inf, -np.inf, np.nan, 2.0 ** -125, 2.0 ** 125, np.nextafter(2.0 ** 125, 0.0)]
    x = np.concatenate([10.0 ** rng.uniform(-307, 308, 400000), rng.uniform(200.0, 6000.0, 200000),
                        rng.uniform(0.25, 4.0, 200000), 1.0 + rng.uniform(-1e-2, 1e-2, 50000), special])
    xt = torch.tensor(x, device="cuda")
    y = rk.eval_exp(xt, 6).cpu().numpy()
    ref = torch.log(xt).cpu().numpy()
    fast = (x >= tiny) & np.isfinite(x)
    bound = np.maximum(3.0 * np.spacing(np.abs(ref[fast])), 2.5e-16)
    assert np.all(np.abs(y[fast] - ref[fast]) <= bound)
    assert y[x == 1.0][0] == 0.0 or abs(y[x == 1.0][0]) < 1e-18
    other = ~fast
    assert np.array_equal(np.isnan(y[other]), np.isnan(ref[other]))
    keep = other & ~np.isnan(ref)
    assert np.array_equal(y[keep], ref[keep])

    xr = np.concatenate([x, -x])
    xrt = torch.tensor(xr, device="cuda")
    yr = rk.eval_exp(xrt, 7).cpu().numpy()
    rr = (1.0 / xrt).cpu().numpy()
    ax = np.abs(xr)
    newton = (ax >= 2.0 ** -125) & (ax < 2.0 ** 125)
    assert np.max(_ulps(yr[newton], rr[newton])) <= 1
    other = ~newton
    assert np.array_equal(np.isnan(yr[other]), np.isnan(rr[other]))
    keep = other & ~np.isnan(rr)
    assert np.array_equal(yr[keep], rr[keep])


def test_cuda_graph_capture_matches_eager(rk):
    """The split step captured once in a CUDA graph and replayed gives the same
    bits as the eager calls."""
    from synth.fields import field_tanh_front

    w, mech = _mech("flame1d")
    m = rk.mech_load(mech)
    _, U0 = field_tanh_front(256, mech.n_species, w.field_seed)
    dx = 1e-2 / 256
    ws = torch.empty(rk.simpler_split_step_workspace_size(m, 256, 4), dtype=torch.uint8, device="cuda")
    Ue = torch.tensor(U0, device="cuda")
    he = torch.zeros(256, dtype=torch.float64, device="cuda")
    for _ in range(3):
        rk.simpler_split_step(m, Ue, w.dt, 1e-4, dx, w.rtol, w.atol, 4, h_cell=he, workspace=ws)
    Ug = torch.tensor(U0, device="cuda")
    hg = torch.zeros(256, dtype=torch.float64, device="cuda")
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s, capture_error_mode="relaxed"):
            rk.simpler_split_step(m, Ug, w.dt, 1e-4, dx, w.rtol, w.atol, 4, h_cell=hg, workspace=ws, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    Ug.copy_(torch.tensor(U0, device="cuda"))
    hg.zero_()
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(Ug, Ue)
    assert torch.equal(hg, he)


def test_autotuner_picks_a_valid_shape(rk, tmp_path):
    from paper_1712_00953_gb300 import autotune
    from synth.fields import initial_state

    w, mech = _mech("small")
    m = rk.mech_load(mech)
    Y = torch.tensor(initial_state(w), device="cuda")
    path = str(tmp_path / "tune.json")
    o = autotune.tune(m, Y, w.dt, w.rtol, w.atol, 4, cache_path=path, reps=1)
    assert (o.lanes_per_cell, o.cells_per_block) in autotune.CANDIDATES
    o2 = autotune.tune(m, Y, w.dt, w.rtol, w.atol, 4, cache_path=path, reps=1)  # cached
    assert (o2.lanes_per_cell, o2.cells_per_block) == (o.lanes_per_cell, o.cells_per_block)
    Y1 = Y.clone()
    rk.rok4e_integrate(m, Y1, w.dt, w.rtol, w.atol, 4, opts=o)
    Y2 = Y.clone()
    rk.rok4e_integrate(m, Y2, w.dt, w.rtol, w.atol, 4)
    torch.cuda.synchronize()
    _assert_state_close(Y1.cpu().numpy(), Y2.cpu().numpy(), mech.n_species, "tuned vs default")
