"""GPU checks of the mixed-precision paths against the FP64 oracle.

Precision level 1 gathers w = nu^T q (in the right-hand side and the
Jacobian-vector product) in double-float on the FP32 pipe, takes the first
Gram-Schmidt pass of Arnoldi with FP32 inner products and the exponentials'
polynomial tails of the rate coefficients in FP32 (the equilibrium constants'
exponentials stay FP64 at every level); level 2 also runs the Jacobian-vector products in
FP32; level 3 keeps the Krylov path in FP64 with a double-float J v core;
level 4 keeps everything FP64 but forms w = nu^T q on the tensor cores from
exact 8-bit digit slices of q; level 5 keeps everything FP64 but the
rate-coefficient exponentials' polynomial tails; level 6 adds an FP32 J v on
FP32 copies of its caches.
The bar is the library's, for every level: |dY| <= 1e-8 + 1e-6 |Y| and
|dT| <= 1e-6 K against the FP64 oracle replaying the GPU run's own step
sequence.
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


def _mech(name):
    from synth.fields import WORKLOADS, mechanism_for

    return WORKLOADS[name], mechanism_for(WORKLOADS[name])


@pytest.mark.parametrize("name", ["small", "mixed"])
def test_mixed_rhs_close_to_oracle(rk, name):
    from oracle.kinetics import Kinetics
    from synth.fields import field_uniform

    w, mech = _mech(name)
    kin = Kinetics(mech)
    U = field_uniform(64, mech.n_species, 13, 500.0, 2500.0)
    m = rk.mech_load(mech)
    out = rk.chem_rhs_mixed(m, torch.tensor(U, device="cuda"), P).cpu().numpy()
    ref = np.array([kin.rhs(u, P) for u in U])
    ns = mech.n_species
    scale = np.max(np.abs(ref[:, :ns]), axis=1, keepdims=True)
    # double-float gather (~2^-44) and FP32 exponential tails (~1e-12)
    assert np.max(np.abs(out[:, :ns] - ref[:, :ns]) / scale) < 1e-10
    assert np.max(np.abs(out[:, ns] - ref[:, ns]) / np.abs(ref[:, ns])) < 1e-10


@pytest.mark.parametrize("name", ["small", "mixed"])
def test_fp32_jvp_close_to_oracle(rk, name):
    from oracle.kinetics import Kinetics
    from synth.fields import field_uniform

    w, mech = _mech(name)
    kin = Kinetics(mech)
    U = field_uniform(48, mech.n_species, 17, 600.0, 2500.0)
    V = np.random.default_rng(2).normal(size=U.shape)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    m = rk.mech_load(mech)
    out = rk.chem_jvp(m, torch.tensor(U, device="cuda"), torch.tensor(V, device="cuda"), P, mode=2).cpu().numpy()
    ref = np.array([kin.jvp(u, P, v) for u, v in zip(U, V)])
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.max(np.abs(out - ref) / scale) < 1e-4


@pytest.mark.parametrize("name", ["small", "flame1d", "batched"])
def test_fp32_jvp_on_fp64_caches_close_to_oracle(rk, name):
    """The J v of precision level 6 (FP32 arithmetic on the FP64 caches,
    rk_chem_jvp mode 5) against the oracle's analytic Jacobian: FP32 rounding
    amplified where forward and reverse rates nearly cancel, the same order
    as the FP32 J v of level 2."""
    from oracle.kinetics import Kinetics
    from synth.fields import field_uniform

    w, mech = _mech(name)
    kin = Kinetics(mech)
    U = field_uniform(48, mech.n_species, 31, 600.0, 2500.0)
    V = np.random.default_rng(9).normal(size=U.shape)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    m = rk.mech_load(mech)
    out = rk.chem_jvp(m, torch.tensor(U, device="cuda"), torch.tensor(V, device="cuda"), P, mode=5).cpu().numpy()
    ref = np.array([kin.jvp(u, P, v) for u, v in zip(U, V)])
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    err = np.max(np.abs(out - ref) / scale)
    print(f"{name}: FP32 J v on the FP64 caches vs oracle {err:.2e} of the row scale")
    assert err < 1e-4


@pytest.mark.parametrize("name", ["small", "flame1d", "batched"])
def test_double_float_jvp_close_to_oracle(rk, name):
    """The J v with its reaction-level core in double-float (precision 3)
    against the oracle's analytic Jacobian: a few 1e-11 of the row scale
    (double-float's ~44-bit significand, amplified where k Pf and kr Pb nearly
    cancel), far inside what the Krylov basis needs (the FP32 J v is ~1e-5)."""
    from oracle.kinetics import Kinetics
    from synth.fields import field_uniform

    w, mech = _mech(name)
    kin = Kinetics(mech)
    U = field_uniform(48, mech.n_species, 19, 600.0, 2500.0)
    V = np.random.default_rng(4).normal(size=U.shape)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    m = rk.mech_load(mech)
    out = rk.chem_jvp(m, torch.tensor(U, device="cuda"), torch.tensor(V, device="cuda"), P, mode=3).cpu().numpy()
    ref = np.array([kin.jvp(u, P, v) for u, v in zip(U, V)])
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.max(np.abs(out - ref) / scale) < 1e-10


@pytest.mark.parametrize("name", ["small", "flame1d", "batched", "adjoint"])
def test_tensor_core_rhs_close_to_oracle(rk, name):
    """w = nu^T q on the tensor cores (precision 4): every q_j is kept down
    to 2^-55 of the cell's largest rate and the rest is exact, so the source
    term meets the FP64 path's own bar against the oracle, with and without
    a source."""
    from oracle.kinetics import Kinetics
    from synth.fields import field_uniform

    w, mech = _mech(name)
    kin = Kinetics(mech)
    U = field_uniform(67, mech.n_species, 23, 300.0, 3000.0)
    src = np.random.default_rng(8).normal(size=U.shape) * 10.0
    m = rk.mech_load(mech)
    Ug = torch.tensor(U, device="cuda")
    for s in (None, src):
        sg = None if s is None else torch.tensor(s, device="cuda")
        out = rk.chem_rhs_tc(m, Ug, P, src=sg).cpu().numpy()
        ref = np.array([kin.rhs(u, P, None if s is None else s[i]) for i, u in enumerate(U)])
        scale = np.max(np.abs(ref), axis=1, keepdims=True)
        err = np.max(np.abs(out - ref) / scale)
        fp64 = rk.chem_rhs(m, Ug, P, src=sg).cpu().numpy()
        print(f"{name}: tensor-core RHS vs oracle {err:.2e} of the row scale; FP64 path "
              f"{np.max(np.abs(fp64 - ref) / scale):.2e}")
        assert err < 1e-11


def test_tensor_core_tiles_that_do_not_fit_are_refused(rk):
    """The 100-species / 500-reaction mechanism's nu^T tiles (7 x 32 of
    them, 112 KiB) fit beside one cell of the point kernel but leave no room
    for a cell of the integrator with M = 4: precision 4 is refused on the
    host with an error, nothing is launched, and the FP64 integration of the
    same cells still runs."""
    w, mech = _mech("adjoint")
    from synth.fields import field_uniform

    U = torch.tensor(field_uniform(4, mech.n_species, 3, 900.0, 1500.0), device="cuda")
    m = rk.mech_load(mech)
    with pytest.raises(rk.RokError, match="shared memory"):
        rk.rok4e_integrate(m, U.clone(), w.dt, w.rtol, w.atol, 4, opts=rk.Opts(precision=4))
    st = torch.zeros(4, 4, dtype=torch.int32, device="cuda")
    rk.rok4e_integrate(m, U, w.dt, w.rtol, w.atol, 4, stats=st)
    torch.cuda.synchronize()
    assert torch.isfinite(U).all() and int(st[:, 3].abs().sum()) == 0


def test_tensor_core_rhs_extreme_cells(rk):
    """Cells whose rates span the widest ranges: 300 K (rates over hundreds
    of orders of magnitude), 3000 K, and cells of one species with every other
    at 1e-30 (nearly every rate tiny beside the few of that species).  The
    digits keep each rate down to 2^-55 of the largest, so the bar against the
    oracle is the FP64 path's."""
    from oracle.kinetics import Kinetics

    w, mech = _mech("batched")
    kin = Kinetics(mech)
    ns = mech.n_species
    rows = []
    for T in (300.0, 3000.0):
        u = np.full(ns + 1, 1.0 / ns)
        u[ns] = T
        rows.append(u)
    for k in range(0, ns, 5):
        u = np.full(ns + 1, 1e-30)
        u[k] = 1.0 - (ns - 1) * 1e-30
        u[ns] = 1400.0
        rows.append(u)
    U = np.array(rows)
    m = rk.mech_load(mech)
    Ug = torch.tensor(U, device="cuda")
    out = rk.chem_rhs_tc(m, Ug, P).cpu().numpy()
    ref = np.array([kin.rhs(u, P) for u in U])
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.all(np.isfinite(out))
    assert np.max(np.abs(out - ref) / scale) < 1e-11


@pytest.mark.parametrize("name", ["small", "flame1d", "batched"])
def test_tensor_core_jvp_close_to_oracle(rk, name):
    """The analytic J v with nu^T dq on the tensor cores (rk_chem_jvp mode
    4) against the oracle's analytic Jacobian, at the FP64 product's bar."""
    from oracle.kinetics import Kinetics
    from synth.fields import field_uniform

    w, mech = _mech(name)
    kin = Kinetics(mech)
    U = field_uniform(40, mech.n_species, 29, 500.0, 2800.0)
    V = np.random.default_rng(6).normal(size=U.shape)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    m = rk.mech_load(mech)
    out = rk.chem_jvp(m, torch.tensor(U, device="cuda"), torch.tensor(V, device="cuda"), P, mode=4).cpu().numpy()
    ref = np.array([kin.jvp(u, P, v) for u, v in zip(U, V)])
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.max(np.abs(out - ref) / scale) < 1e-10


def _run(rk, mech, U, w, precision, cap=8192, M=4):
    m = rk.mech_load(mech)
    Y = torch.tensor(U, device="cuda")
    n = U.shape[0]
    st = torch.zeros(n, 4, dtype=torch.int32, device="cuda")
    tr = torch.zeros(n, cap, dtype=torch.float64, device="cuda")
    rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, M, stats=st, opts=rk.Opts(precision=precision, trace=tr))
    torch.cuda.synchronize()
    return Y.cpu().numpy(), st.cpu().numpy(), tr.cpu().numpy()


@pytest.mark.parametrize("precision", [1, 2, 3, 4, 5, 6])
def test_mixed_integration_error_vs_fp64_oracle(rk, precision):
    """Mixed-precision ROK4E on the small workload (10 species / 24
    reactions, one 1e-6 s step), replayed through the FP64 oracle, at the
    library's bar: |dY| <= 1e-8 + 1e-6 |Y|, |dT| <= 1e-6 K."""
    from oracle import rok4e as orok
    from oracle.kinetics import Kinetics
    from synth.fields import initial_state

    w, mech = _mech("small")
    U = initial_state(w)[::8]
    out, st, tr = _run(rk, mech, U, w, precision)
    assert np.all(st[:, 3] == 0)
    ref, _ = orok.integrate_cells(Kinetics(mech), U, P, w.dt, w.rtol, w.atol, 4,
                                  replay=[[(abs(h), h > 0) for h in r if h != 0.0] for r in tr])
    ns = mech.n_species
    dY = np.abs(out[:, :ns] - ref[:, :ns])
    dT = np.abs(out[:, ns] - ref[:, ns])
    excess = dY - (1e-8 + 1e-6 * np.abs(ref[:, :ns]))
    print(f"mixed level {precision} vs FP64 oracle (replay): max |dY| {dY.max():.3e}, max |dT| {dT.max():.3e} K")
    assert excess.max() <= 0.0, excess.max()
    assert dT.max() <= 1e-6, dT.max()


@pytest.mark.parametrize("precision", [0, 1, 2, 3, 4, 5, 6])
def test_flame_mechanism_levels_vs_fp64_oracle(rk, precision):
    """The precision levels on the 1-D flame's mechanism (30 species / 150
    reactions, 4 third-body, 2 Troe) and tanh field: the reaction sub-step of
    the first Simpler split step (constant source T(U_n), dt = 1e-7 s) over
    all 2048 points, and on 24 of them -- the 8 that took the most attempts
    and 16 spread over the grid -- the oracle replaying each point's recorded
    step sequence with the same source.  Bar |dY| <= 1e-8 + 1e-6 |Y|,
    |dT| <= 1e-6 K; the per-species maxima are printed."""
    from oracle import rok4e as orok
    from oracle import splitting as osp
    from oracle.kinetics import Kinetics
    from synth.fields import field_tanh_front

    w, mech = _mech("mixed")
    npts = 2048
    _, U0 = field_tanh_front(npts, mech.n_species, w.field_seed)
    src = osp.diffusion_op(U0, 1e-4, 1e-2 / npts)
    m = rk.mech_load(mech)
    Y = torch.tensor(U0, device="cuda")
    st = torch.zeros(npts, 4, dtype=torch.int32, device="cuda")
    tr = torch.zeros(npts, 512, dtype=torch.float64, device="cuda")
    rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, 4, src=torch.tensor(src, device="cuda"), stats=st,
                       opts=rk.Opts(precision=precision, trace=tr))
    torch.cuda.synchronize()
    out, st, tr = Y.cpu().numpy(), st.cpu().numpy(), tr.cpu().numpy()
    assert np.all(st[:, 3] == 0)
    att = st[:, 0] + st[:, 1]
    assert att.max() < 512
    hot = list(np.argsort(-att, kind="stable")[:8])
    spread = [int(i * 0.6180339887498949 * npts) % npts for i in range(1, 40)]
    cells = hot + [c for c in spread if c not in hot][:16]
    ref, _ = orok.integrate_cells(Kinetics(mech), U0[cells], P, w.dt, w.rtol, w.atol, 4, src=src[cells],
                                  replay=[[(abs(h), h > 0) for h in tr[c] if h != 0.0] for c in cells])
    ns = mech.n_species
    dY = np.abs(out[cells, :ns] - ref[:, :ns])
    dT = np.abs(out[cells, ns] - ref[:, ns])
    excess = dY - (1e-8 + 1e-6 * np.abs(ref[:, :ns]))
    print(f"flame mechanism, precision {precision} vs FP64 oracle (replay, {len(cells)} points, up to "
          f"{att.max()} attempts): max |dY| {dY.max():.3e}, max |dT| {dT.max():.3e} K; per species max |dY| "
          f"{np.array2string(dY.max(axis=0), precision=1)}")
    assert excess.max() <= 0.0, excess.max()
    assert dT.max() <= 1e-6, dT.max()


def test_mixed_split_steps_vs_fp64_gpu(rk):
    """Mixed and FP64 Simpler split steps on the 1-D workload's field: the
    per-species difference after 5 steps stays at the level of the adaptive
    integrator's own tolerance."""
    from synth.fields import field_tanh_front

    w, mech = _mech("mixed")
    m = rk.mech_load(mech)
    _, U0 = field_tanh_front(512, mech.n_species, w.field_seed)
    dx = 1e-2 / 512
    res = {}
    for prec in (0, 1, 2, 3, 4, 5, 6):
        U = torch.tensor(U0, device="cuda")
        hc = torch.zeros(512, dtype=torch.float64, device="cuda")
        for _ in range(5):
            rk.simpler_split_step(m, U, w.dt, 1e-4, dx, w.rtol, w.atol, 4, h_cell=hc,
                                  opts=rk.Opts(precision=prec))
        torch.cuda.synchronize()
        res[prec] = U.cpu().numpy()
    ns = mech.n_species
    for prec in (1, 2, 3, 4, 5, 6):
        dY = np.abs(res[prec][:, :ns] - res[0][:, :ns])
        dT = np.abs(res[prec][:, ns] - res[0][:, ns])
        print(f"mixed level {prec} vs FP64 GPU after 5 split steps: max |dY| {dY.max():.3e} (per species "
              f"{np.array2string(dY.max(axis=0), precision=1)}), max |dT| {dT.max():.3e} K")
        assert np.all(np.isfinite(res[prec]))
        assert dY.max() < 1e-6 and dT.max() < 1e-3


@pytest.mark.parametrize("precision", [5, 6])
def test_batched_mechanism_levels_vs_fp64_oracle(rk, precision):
    """Precision 5 (FP32 exponential tails only) and 6 (also an FP32 J v on
    the FP64 caches) on the batched workload's
    mechanism and field (53 species / 325 reactions, one 1e-6 s step of 64
    cells spread over the 2^20-cell field), replayed through the FP64 oracle
    at the library's bar."""
    from oracle import rok4e as orok
    from oracle.kinetics import Kinetics
    from synth.fields import initial_state

    w, mech = _mech("batched")
    U_all = initial_state(w, n_cells=1 << 14)
    U = U_all[np.linspace(0, U_all.shape[0] - 1, 24).astype(np.int64)]
    out, st, tr = _run(rk, mech, U, w, precision)
    assert np.all(st[:, 3] == 0)
    ref, _ = orok.integrate_cells(Kinetics(mech), U, P, w.dt, w.rtol, w.atol, 4,
                                  replay=[[(abs(h), h > 0) for h in r if h != 0.0] for r in tr])
    ns = mech.n_species
    dY = np.abs(out[:, :ns] - ref[:, :ns])
    dT = np.abs(out[:, ns] - ref[:, ns])
    print(f"batched mechanism, precision {precision} vs FP64 oracle (replay): max |dY| {dY.max():.3e}, "
          f"max |dT| {dT.max():.3e} K")
    assert np.all(dY <= 1e-8 + 1e-6 * np.abs(ref[:, :ns]))
    assert dT.max() <= 1e-6


@pytest.mark.parametrize("lanes", [8, 16])
def test_level_6_with_fewer_lanes_per_cell(rk, lanes):
    """Precision 6 with 8 and 16 lanes per cell (the FP32 J v's reductions
    and cache copies over smaller groups) on the small workload, replayed
    through the FP64 oracle at the library's bar."""
    from oracle import rok4e as orok
    from oracle.kinetics import Kinetics
    from synth.fields import initial_state

    w, mech = _mech("small")
    U = initial_state(w)[::8]
    m = rk.mech_load(mech)
    Y = torch.tensor(U, device="cuda")
    n = U.shape[0]
    st = torch.zeros(n, 4, dtype=torch.int32, device="cuda")
    tr = torch.zeros(n, 8192, dtype=torch.float64, device="cuda")
    rk.rok4e_integrate(m, Y, w.dt, w.rtol, w.atol, 4, stats=st,
                       opts=rk.Opts(precision=6, lanes_per_cell=lanes, trace=tr))
    torch.cuda.synchronize()
    out, st, tr = Y.cpu().numpy(), st.cpu().numpy(), tr.cpu().numpy()
    assert np.all(st[:, 3] == 0)
    ref, _ = orok.integrate_cells(Kinetics(mech), U, P, w.dt, w.rtol, w.atol, 4,
                                  replay=[[(abs(h), h > 0) for h in r if h != 0.0] for r in tr])
    ns = mech.n_species
    assert np.all(np.abs(out[:, :ns] - ref[:, :ns]) <= 1e-8 + 1e-6 * np.abs(ref[:, :ns]))
    assert np.max(np.abs(out[:, ns] - ref[:, ns])) <= 1e-6
