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
    """Bitwise equality with rk_simpler_split_step (both run the same kernels on
    the same inputs, and a cell's bits do not depend on where its scratch lies).
    A first call with the 53-species mechanism on 2048 points leaves different
    contents at different offsets of the static array, so leftovers that should
    have been cleared would show in the 512-point calls that follow."""
    from paper_1712_00953_gb300._native import RkOpts
    from synth.fields import WORKLOADS, field_tanh_front, mechanism_for

    opts = RkOpts()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    dt, D, M = 1e-7, 1e-4, 4

    mech_big = mechanism_for(WORKLOADS["batched"])
    hbig = _load_mech(lib, mech_big)
    _, Ubig = field_tanh_front(2048, mech_big.n_species, 7)
    Ug = torch.tensor(Ubig, device="cuda")
    hg = torch.zeros(2048, dtype=torch.float64, device="cuda")
    rc = lib.rk_simpler_split_step_noalloc(hbig, _ptr(Ug), _ptr(hg), 2048, 101325.0, dt, D, 1e-2 / 2048, 1e-6,
                                           1e-10, M, ctypes.byref(opts), None, stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert torch.isfinite(Ug).all()

    w = WORKLOADS["flame1d"]
    mech = mechanism_for(w)
    h = _load_mech(lib, mech)
    npts = 512
    _, U0 = field_tanh_front(npts, mech.n_species, w.field_seed)
    dx = 1e-2 / npts
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
        assert torch.equal(Ua, Ub), call
        assert torch.equal(sa, sb), call
        assert torch.equal(ha, hb), call
    assert lib.rk_mech_free(h) == 0
    assert lib.rk_mech_free(hbig) == 0


def test_noalloc_rejects_sizes_beyond_the_static_scratch(lib):
    from paper_1712_00953_gb300 import _native
    from paper_1712_00953_gb300._native import RkOpts
    from synth.fields import WORKLOADS, mechanism_for

    mech = mechanism_for(WORKLOADS["flame1d"])
    h = _load_mech(lib, mech)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    U = torch.zeros(1, dtype=torch.float64, device="cuda")
    # 5606 points x 31 values is one point beyond the 4 MiB scratch; nothing is launched
    rc = lib.rk_simpler_split_step_noalloc(h, _ptr(U), None, 5606, 101325.0, 1e-7, 1e-4, 1e-5, 1e-6, 1e-10, 4,
                                           ctypes.byref(RkOpts()), None, stream)
    assert rc == -4
    msg = _native.last_error(lib)
    assert "static scratch" in msg and "at most 5605 points" in msg, msg
    assert lib.rk_mech_free(h) == 0
