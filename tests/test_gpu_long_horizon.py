"""The 1-D flame over its full horizon: 1000 Simpler split steps of 1e-7 s
(Eq. simpler_balanced) on the GPU, checked against the C oracle.

* Full size (2048 points, 30 species / 150 reactions): all 1000 split steps run
  on the GPU in the benchmark's launch configuration (carried step sizes,
  static-bin queue, 8 cells per block).  At steps 0, 100, ..., 900 and 999 the
  GPU's input state and every point's recorded step sequence are kept; the C
  oracle then takes that same split step from the GPU's own state over the
  whole grid, replaying the recorded sequences.  Bar at every point:
  |dY| <= 1e-8 + 1e-6 |Y|, |dT| <= 1e-6 K.
* Accumulated error: the same front on 128 points, 1000 split steps on the
  GPU and, end to end from the initial field, by the C oracle replaying every
  step's recorded sequences.  The final states meet the same bar; the final
  error is printed.
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
    worst = []
    for s, U_in, h_in, trs, U_out, h_out in kept:
        ref, h_ref, st_ref = co.simpler_steps(U_in, h_in, 1, w.dt, D, dx, w.rtol, w.atol, 4, replay=trs[None])
        excess, dY, dT = _bar(U_out, ref, ns)
        worst.append((s, dY, dT))
        print(f"split step {s}: max |dY| {dY:.3e}, max |dT| {dT:.3e} K, T max {U_out[:, ns].max():.1f} K")
        assert excess <= 0.0, (s, excess)
        assert dT <= 1e-6, (s, dT)
        assert np.max(np.abs(h_out - h_ref) / h_ref) < 1e-5, s
    print("worst over the checkpoints:", max(x[1] for x in worst), max(x[2] for x in worst))


def test_coarse_grid_1000_steps_end_to_end(rk, flame):
    from synth.fields import field_tanh_front

    w, mech, co = flame
    npts = 128
    _, U0 = field_tanh_front(npts, mech.n_species, w.field_seed)
    dx = 1e-2 / npts
    m = rk.mech_load(mech)
    U = torch.tensor(U0, device="cuda")
    hc = torch.zeros(npts, dtype=torch.float64, device="cuda")
    ws = torch.empty(rk.simpler_split_step_workspace_size(m, npts, 4), dtype=torch.uint8, device="cuda")
    st = torch.zeros(NSTEPS, npts, 4, dtype=torch.int32, device="cuda")
    tr = torch.zeros(NSTEPS, npts, CAP, dtype=torch.float64, device="cuda")
    for s in range(NSTEPS):
        rk.simpler_split_step(m, U, w.dt, D, dx, w.rtol, w.atol, 4, h_cell=hc, stats=st[s],
                              opts=rk.Opts(trace=tr[s]), workspace=ws)
    torch.cuda.synchronize()
    s_np = st.cpu().numpy()
    assert np.all(s_np[:, :, 3] == 0)
    assert (s_np[:, :, 0] + s_np[:, :, 1]).max() < CAP
    ref, _, _ = co.simpler_steps(U0, np.zeros(npts), NSTEPS, w.dt, D, dx, w.rtol, w.atol, 4,
                                 replay=tr.cpu().numpy())
    gpu = U.cpu().numpy()
    ns = mech.n_species
    excess, dY, dT = _bar(gpu, ref, ns)
    print(f"128 points after {NSTEPS} split steps (t = {NSTEPS * w.dt:.1e} s): max |dY| {dY:.3e}, "
          f"max |dT| {dT:.3e} K; T from {U0[:, ns].min():.0f}..{U0[:, ns].max():.0f} to "
          f"{gpu[:, ns].min():.0f}..{gpu[:, ns].max():.0f} K; {int(s_np[:, :, 0].sum())} substeps")
    assert excess <= 0.0, excess
    assert dT <= 1e-6, dT
