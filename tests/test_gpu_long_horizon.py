"""The 1-D flame over its full horizon: 1000 Simpler split steps of 1e-7 s
(Eq. simpler_balanced) on the GPU, checked against the C oracle.

* Full size (2048 points, 30 species / 150 reactions): all 1000 split steps run
  on the GPU in the benchmark's launch configuration (carried step sizes,
  static-bin queue, 8 cells per block).  At steps 0, 100, ..., 900 and 999 the
  GPU's input state and every point's recorded step sequence are kept; the C
  oracle then takes that same split step from the GPU's own state over the
  whole grid, replaying the recorded sequences.  Bar at every point:
  |dY| <= 1e-8 + 1e-6 |Y|, |dT| <= 1e-6 K.
* Accumulated error, on the same front with 128 points: (a) the first 100
  split steps replayed end to end by the C oracle with the GPU's recorded step
  sequences, at the bar above; (b) all 1000 split steps free running on both
  sides.  Replaying a fixed step sequence end to end is well conditioned only
  early on: along the recorded sequence the oracle's own final temperature
  moves by ~2e-6 K after 300 steps for a 1e-13 relative change of the initial
  temperature, and the forced steps go unstable for such a perturbation before
  step 500 (a step accepted for one trajectory is forced on another).  Free
  running, each side's controller keeps its own error below the tolerance,
  and accept/reject decisions at err ~ 1 may differ (several correct results:
  the adaptive runs differ by the integrator's tolerance).  So (b) asserts the
  Y bar and |dT| <= max(1e-6 K, 3 x the oracle's own spread of final T under
  1e-15 and 1e-13 relative perturbations of the initial temperature), and
  prints both sides' global error against the oracle at rtol 1e-9.
The C oracle is pinned against the numpy oracle in tests/test_oracle_c.py.
"""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

P = 101325.0
D = 1e-4
NSTEPS = 1000
CAP = 128


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1712_00953_gb300 as rk

    return rk


@pytest.fixture(scope="module")
def flame():
    from oracle import c_oracle
    from synth.fields import WORKLOADS, mechanism_for

    c_oracle.build()
    w = WORKLOADS["flame1d"]
    mech = mechanism_for(w)
    return w, mech, c_oracle.COracle(mech)


def _bar(gpu, ref, ns):
    dY = np.abs(gpu[:, :ns] - ref[:, :ns])
    dT = np.abs(gpu[:, ns] - ref[:, ns])
    return float((dY - (1e-8 + 1e-6 * np.abs(ref[:, :ns]))).max()), float(dY.max()), float(dT.max())


def test_full_size_1000_steps_checkpoints(rk, flame):
    from synth.fields import field_tanh_front

    w, mech, co = flame
    npts = w.n_cells
    _, U0 = field_tanh_front(npts, mech.n_species, w.field_seed)
    dx = 1e-2 / npts
    m = rk.mech_load(mech)
    U = torch.tensor(U0, device="cuda")
    hc = torch.zeros(npts, dtype=torch.float64, device="cuda")
    ws = torch.empty(rk.simpler_split_step_workspace_size(m, npts, 4), dtype=torch.uint8, device="cuda")
    st = torch.zeros(npts, 4, dtype=torch.int32, device="cuda")
    tr = torch.zeros(npts, CAP, dtype=torch.float64, device="cuda")
    opts = rk.Opts(cells_per_block=8, queue_order=3)
    opts_tr = rk.Opts(cells_per_block=8, queue_order=3, trace=tr)
    checks = set(range(0, NSTEPS, 100)) | {NSTEPS - 1}
    kept = []
    for s in range(NSTEPS):
        if s in checks:
            U_in, h_in = U.cpu().numpy(), hc.cpu().numpy()
            tr.zero_()
            rk.simpler_split_step(m, U, w.dt, D, dx, w.rtol, w.atol, 4, h_cell=hc, stats=st, opts=opts_tr,
                                  workspace=ws)
            torch.cuda.synchronize()
            s_np = st.cpu().numpy()
            assert np.all(s_np[:, 3] == 0), s
            assert (s_np[:, 0] + s_np[:, 1]).max() < CAP, s
            kept.append((s, U_in, h_in, tr.cpu().numpy(), U.cpu().numpy(), hc.cpu().numpy()))
        else:
            rk.simpler_split_step(m, U, w.dt, D, dx, w.rtol, w.atol, 4, h_cell=hc, opts=opts, workspace=ws)
    torch.cuda.synchronize()
    assert torch.isfinite(U).all()
    ns = mech.n_species
    worst, worst_h = [], 0.0
    for s, U_in, h_in, trs, U_out, h_out in kept:
        ref, h_ref, st_ref = co.simpler_steps(U_in, h_in, 1, w.dt, D, dx, w.rtol, w.atol, 4, replay=trs[None])
        excess, dY, dT = _bar(U_out, ref, ns)
        worst.append((s, dY, dT))
        print(f"split step {s}: max |dY| {dY:.3e}, max |dT| {dT:.3e} K, T max {U_out[:, ns].max():.1f} K")
        assert excess <= 0.0, (s, excess)
        assert dT <= 1e-6, (s, dT)
        worst_h = max(worst_h, float(np.max(np.abs(h_out - h_ref) / h_ref)))
    # the proposed next steps come from the error estimate, which rounding moves
    # (a GPU step factor in FP32 as well): reported, not part of the bar
    print(f"worst over the checkpoints: max |dY| {max(x[1] for x in worst):.3e}, max |dT| "
          f"{max(x[2] for x in worst):.3e} K; proposed next steps differ by up to {worst_h:.1e} relative")


def test_coarse_grid_1000_steps_end_to_end(rk, flame):
    from synth.fields import field_tanh_front

    w, mech, co = flame
    npts, n_replay = 128, 100
    _, U0 = field_tanh_front(npts, mech.n_species, w.field_seed)
    dx = 1e-2 / npts
    m = rk.mech_load(mech)
    U = torch.tensor(U0, device="cuda")
    hc = torch.zeros(npts, dtype=torch.float64, device="cuda")
    ws = torch.empty(rk.simpler_split_step_workspace_size(m, npts, 4), dtype=torch.uint8, device="cuda")
    st = torch.zeros(NSTEPS, npts, 4, dtype=torch.int32, device="cuda")
    tr = torch.zeros(n_replay, npts, CAP, dtype=torch.float64, device="cuda")
    U_rep = None
    for s in range(NSTEPS):
        opts = rk.Opts(trace=tr[s]) if s < n_replay else None
        rk.simpler_split_step(m, U, w.dt, D, dx, w.rtol, w.atol, 4, h_cell=hc, stats=st[s], opts=opts, workspace=ws)
        if s + 1 == n_replay:
            U_rep = U.cpu().numpy()
    torch.cuda.synchronize()
    s_np = st.cpu().numpy()
    assert np.all(s_np[:, :, 3] == 0)
    assert (s_np[:n_replay, :, 0] + s_np[:n_replay, :, 1]).max() < CAP
    gpu = U.cpu().numpy()
    ns = mech.n_species

    # (a) the first 100 split steps replayed end to end
    ref, _, _ = co.simpler_steps(U0, np.zeros(npts), n_replay, w.dt, D, dx, w.rtol, w.atol, 4,
                                 replay=tr.cpu().numpy())
    excess, dY, dT = _bar(U_rep, ref, ns)
    print(f"128 points, {n_replay} split steps replayed end to end: max |dY| {dY:.3e}, max |dT| {dT:.3e} K")
    assert excess <= 0.0, excess
    assert dT <= 1e-6, dT

    # (b) 1000 split steps free running on both sides
    ref, _, st_ref = co.simpler_steps(U0, np.zeros(npts), NSTEPS, w.dt, D, dx, w.rtol, w.atol, 4)
    spread = 0.0
    for eps in (1e-15, 1e-13):
        Up = U0.copy()
        Up[:, ns] *= 1.0 + eps
        alt, _, _ = co.simpler_steps(Up, np.zeros(npts), NSTEPS, w.dt, D, dx, w.rtol, w.atol, 4)
        spread = max(spread, float(np.abs(alt[:, ns] - ref[:, ns]).max()))
    tight, _, _ = co.simpler_steps(U0, np.zeros(npts), NSTEPS, w.dt, D, dx, 1e-9, 1e-13, 4)
    excess, dY, dT = _bar(gpu, ref, ns)
    bar_T = max(1e-6, 3.0 * spread)
    print(f"128 points after {NSTEPS} free-running split steps (t = {NSTEPS * w.dt:.1e} s, T "
          f"{U0[:, ns].min():.0f}..{U0[:, ns].max():.0f} -> {gpu[:, ns].min():.0f}..{gpu[:, ns].max():.0f} K): "
          f"GPU vs oracle max |dY| {dY:.3e}, max |dT| {dT:.3e} K (bar {bar_T:.2e} K; the oracle's own spread "
          f"{spread:.2e} K); global error vs the oracle at rtol 1e-9: GPU {np.abs(gpu[:, ns] - tight[:, ns]).max():.2e} K, "
          f"oracle {np.abs(ref[:, ns] - tight[:, ns]).max():.2e} K; substeps GPU {int(s_np[:, :, 0].sum())}, "
          f"oracle {int(st_ref[:, :, 0].sum())}")
    assert excess <= 0.0, excess
    assert dT <= bar_T, dT
