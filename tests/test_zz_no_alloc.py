"""The allocation-free split step (rk_simpler_split_step_noalloc) against the
workspace version, called through the C ABI.

Callers that cannot allocate device memory while stepping (fixed memory pools,
host codes without a CUDA allocator) use the entry point that keeps its scratch
in a static device array; this checks that it reproduces
rk_simpler_split_step on two calls in a row, i.e. that the scratch the second
call inherits from the first does not leak into its result.  The file name
makes pytest collect it last.
"""

import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_00953_gb300 import _native

    return _native.load()


def _load_mech(lib, mech):
    from paper_1712_00953_gb300._native import RkMechDesc

    arrs = [np.ascontiguousarray(getattr(mech, k), dtype=dt) for k, dt in
            (("elem", np.int32), ("W", np.float64), ("nasa", np.float64), ("rxn_sp", np.int32),
             ("rxn_nu", np.int32), ("arrh", np.float64), ("reversible", np.uint8), ("kind", np.int32),
             ("eff", np.float64), ("falloff", np.float64))]
    d = RkMechDesc(mech.n_species, mech.n_reactions, *(a.ctypes.data for a in arrs))
    h = ctypes.c_void_p()
    assert lib.rk_mech_load(ctypes.byref(d), ctypes.byref(h)) == 0
    return h


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_split_step_matches_workspace_version(lib):
    from paper_1712_00953_gb300._native import RkOpts
    from synth.fields import WORKLOADS, field_tanh_front, mechanism_for

    w = WORKLOADS["flame1d"]
    mech = mechanism_for(w)
    h = _load_mech(lib, mech)
    npts = 512
    _, U0 = field_tanh_front(npts, mech.n_species, w.field_seed)
    dx, D, M = 1e-2 / npts, 1e-4, 4
    opts = RkOpts()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    Ua = torch.tensor(U0, device="cuda")
    ha = torch.zeros(npts, dtype=torch.float64, device="cuda")
    nb = lib.rk_simpler_split_step_workspace_size(h, npts, M, ctypes.byref(opts))
    ws = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    Ub = torch.tensor(U0, device="cuda")
    hb = torch.zeros(npts, dtype=torch.float64, device="cuda")
    sa = torch.zeros(npts, 4, dtype=torch.int32, device="cuda")
    sb = torch.zeros(npts, 4, dtype=torch.int32, device="cuda")
    for call in range(2):  # two calls in a row: the second inherits the scratch of the first
        rc = lib.rk_simpler_split_step(h, _ptr(Ua), _ptr(ha), npts, 101325.0, w.dt, D, dx, w.rtol, w.atol, M,
                                       ctypes.byref(opts), _ptr(sa), _ptr(ws), nb, stream)
        assert rc == 0
        rc = lib.rk_simpler_split_step_noalloc(h, _ptr(Ub), _ptr(hb), npts, 101325.0, w.dt, D, dx, w.rtol,
                                               w.atol, M, ctypes.byref(opts), _ptr(sb), stream)
        assert rc == 0
        torch.cuda.synchronize()
        a, b = Ua.cpu().numpy(), Ub.cpu().numpy()
        ns = mech.n_species
        # the tolerance of the parity tests: |dY| <= 1e-8 + 1e-6 |Y|, |dT| <= 1e-6 K
        assert np.all(np.abs(b[:, :ns] - a[:, :ns]) <= 1e-8 + 1e-6 * np.abs(a[:, :ns])), call
        assert np.all(np.abs(b[:, ns] - a[:, ns]) <= 1e-6), call
        assert torch.equal(sa, sb)
        assert torch.equal(ha, hb)
    assert lib.rk_mech_free(h) == 0


def test_noalloc_rejects_sizes_beyond_the_static_scratch(lib):
    from paper_1712_00953_gb300 import _native
    from paper_1712_00953_gb300._native import RkOpts
    from synth.fields import WORKLOADS, mechanism_for

    mech = mechanism_for(WORKLOADS["flame1d"])
    h = _load_mech(lib, mech)
    npts = 200000  # x 31 values is beyond the 4 MiB scratch; nothing is launched
    U = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = lib.rk_simpler_split_step_noalloc(h, _ptr(U), None, npts, 101325.0, 1e-7, 1e-4, 1e-5, 1e-6, 1e-10, 4,
                                           ctypes.byref(RkOpts()), None,
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -4
    assert "static scratch" in _native.last_error(lib)
    assert lib.rk_mech_free(h) == 0
