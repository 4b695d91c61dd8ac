"""GB300 ROK4E reaction step and Simpler balanced splitting (arXiv:1712.00953).

Thin Python binding over the C ABI of ``librok4e.so`` (include/rok4e.h).  The
functions keep the C names without the ``rk_`` prefix and only marshal
arguments: tensors must be contiguous float64 CUDA tensors; every step of the
computation runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  The library is loaded on first use; every call raises
ImportError if it has not been built (there is no fallback path).
"""

from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native
from ._native import RkMechDesc, RkOpts

_LIB = None


def _L():
    global _LIB
    if _LIB is None:
        _LIB = _native.load()
    return _LIB

__all__ = ["Mechanism", "mech_load", "mech_validate", "chem_rhs", "chem_rhs_mixed", "chem_rhs_tc", "simpler_split_step_ext", "chem_rhs_cv", "chem_jvp_cv",
           "chem_jvp", "rok4e_integrate", "rkdp_integrate", "chem_rhs_aux", "chem_jvp_aux", "AUX_EXTRA",
           "rok4e_workspace_size", "simpler_split_step", "simpler_split_step_workspace_size",
           "diffusion_1d", "diffusion_1d_ghost", "ssprk3_stage_ghost", "GhostTransport",
           "simpler_split_step_phases", "halo_exchange", "simpler_split_step_sharded", "probe_throughput", "eval_exp", "split_step", "SCHEMES", "rok4e_fixed_steps",
           "rok4e_adjoint", "rok4e_adjoint_workspace_size", "FixedStepROK4E", "Opts", "RokError", "STATS_FIELDS"]

STATS_FIELDS = ("n_accept", "n_reject", "n_rhs", "status")


class RokError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        msg = _native.last_error(_L())
        raise RokError(f"{what}: {_L().rk_status_string(rc).decode()} ({rc}): {msg}")


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t, name, n_elems=None, dtype=torch.float64):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} CUDA tensor")
    if n_elems is not None and t.numel() < n_elems:
        raise ValueError(f"{name} has {t.numel()} elements, needs {n_elems}")
    return ctypes.c_void_p(t.data_ptr())


class _HostDesc:
    """Keeps the numpy arrays of a description alive while the C call reads them."""

    def __init__(self, mech):
        self.arrays = dict(
            elem=np.ascontiguousarray(mech.elem, dtype=np.int32),
            W=np.ascontiguousarray(mech.W, dtype=np.float64),
            nasa=np.ascontiguousarray(mech.nasa, dtype=np.float64),
            rxn_sp=np.ascontiguousarray(mech.rxn_sp, dtype=np.int32),
            rxn_nu=np.ascontiguousarray(mech.rxn_nu, dtype=np.int32),
            arrh=np.ascontiguousarray(mech.arrh, dtype=np.float64),
            reversible=np.ascontiguousarray(mech.reversible, dtype=np.uint8),
            kind=np.ascontiguousarray(mech.kind, dtype=np.int32),
            eff=np.ascontiguousarray(mech.eff, dtype=np.float64),
            falloff=np.ascontiguousarray(mech.falloff, dtype=np.float64),
        )
        a = self.arrays
        self.desc = RkMechDesc(int(mech.W.shape[0]), int(mech.arrh.shape[0]),
                               *(a[k].ctypes.data for k in ("elem", "W", "nasa", "rxn_sp", "rxn_nu", "arrh",
                                                            "reversible", "kind", "eff", "falloff")))


def mech_validate(mech) -> str:
    """Host-only validation; returns '' when valid, else the reason."""
    hd = _HostDesc(mech)
    buf = ctypes.create_string_buffer(512)
    rc = _L().rk_mech_validate(ctypes.byref(hd.desc), buf, 512)
    return "" if rc == 0 else buf.value.decode(errors="replace")


class Mechanism:
    """A mechanism uploaded to the current CUDA device (rk_mech_load)."""

    def __init__(self, mech):
        hd = _HostDesc(mech)
        h = ctypes.c_void_p()
        _check(_L().rk_mech_load(ctypes.byref(hd.desc), ctypes.byref(h)), "rk_mech_load")
        self.handle = h
        self.n_species = int(mech.W.shape[0])
        self.n_reactions = int(mech.arrh.shape[0])
        self.n_state = self.n_species + 1

    def info(self):
        ns, nr, nb = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t()
        _check(_L().rk_mech_info(self.handle, ctypes.byref(ns), ctypes.byref(nr), ctypes.byref(nb)), "rk_mech_info")
        return ns.value, nr.value, nb.value

    def free(self):
        if self.handle:
            _L().rk_mech_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mech_load(mech) -> Mechanism:
    return Mechanism(mech)


class Opts:
    """Integration options (rk_opts); None fields keep the library defaults."""

    def __init__(self, jv_mode=0, max_attempts=0, lanes_per_cell=0, cells_per_block=0, h0=0.0, fixed_h=0.0,
                 trace=None, events=None, precision=0, queue_order=0, blocks_per_sm=0, rho_cell=None,
                 reactor=None):
        self.jv_mode, self.max_attempts = jv_mode, max_attempts
        self.lanes_per_cell, self.cells_per_block = lanes_per_cell, cells_per_block
        self.h0, self.fixed_h = h0, fixed_h
        self.trace = trace  # CUDA float64 tensor [ncell, cap] or None
        self.events = events  # (begin, end) torch.cuda.Event pair around the integration kernel
        # rk_opts.precision: 0 FP64; 1 double-float nu^T q, FP32 first
        # Gram-Schmidt products and rate-coefficient exp tails; 2 as 1 with an
        # FP32 J v; 3 FP64 Krylov path, double-float J v core, FP32 exp tails;
        # 4 nu^T q on the tensor cores; 5 FP32 rate-coefficient exp tails only;
        # 6 as 5 with an FP32 J v on FP32 copies of its caches
        self.precision = precision
        self.queue_order, self.blocks_per_sm = queue_order, blocks_per_sm
        self.rho_cell = rho_cell  # CUDA float64 [ncell]: constant-volume cells of these densities
        # 0 constant pressure, 1 constant volume (implied by rho_cell), 2 conservative
        # variables with the auxiliary temperature (rows of n_species + 1 + AUX_EXTRA)
        self.reactor = reactor if reactor is not None else (0 if rho_cell is None else 1)

    def c(self):
        cap = 0 if self.trace is None else int(self.trace.shape[-1])
        tp = None if self.trace is None else _dptr(self.trace, "trace")
        eb = ee = None
        if self.events is not None:
            eb, ee = (ctypes.c_void_p(e.cuda_event) for e in self.events)
        rc = None if self.rho_cell is None else _dptr(self.rho_cell, "rho_cell")
        return RkOpts(self.jv_mode, self.max_attempts, self.lanes_per_cell, self.cells_per_block, self.h0,
                      self.fixed_h, cap, self.precision, tp, eb, ee, self.queue_order, self.blocks_per_sm,
                      int(self.reactor), 0, rc)


AUX_EXTRA = 5  # rho, rho v (3), rho E after T in the auxiliary-temperature rows


def _ncell(Y, m, extra=0):
    if Y.dim() != 2 or Y.shape[1] != m.n_state + extra:
        raise ValueError(f"state must be [ncell, {m.n_state + extra}]")
    return int(Y.shape[0])


def _extra(opts):
    return AUX_EXTRA if opts is not None and opts.reactor == 2 else 0


def chem_rhs_aux(m: Mechanism, U, src=None, out=None, stream=None):
    """dU/dt of the auxiliary-temperature system (rk_chem_rhs_aux); rows
    [rho Y (Ns), T, rho, rho v (3), rho E]."""
    n = _ncell(U, m, AUX_EXTRA)
    out = torch.empty_like(U) if out is None else out
    _check(_L().rk_chem_rhs_aux(m.handle, _dptr(U, "U"), _dptr(src, "src", U.numel()),
                                _dptr(out, "out", U.numel()), n, _stream_ptr(stream)), "rk_chem_rhs_aux")
    return out


def chem_jvp_aux(m: Mechanism, U, V, src=None, mode=0, out=None, stream=None):
    n = _ncell(U, m, AUX_EXTRA)
    out = torch.empty_like(U) if out is None else out
    _check(_L().rk_chem_jvp_aux(m.handle, _dptr(U, "U"), _dptr(src, "src", U.numel()), _dptr(V, "V", U.numel()),
                                _dptr(out, "out", U.numel()), n, int(mode), _stream_ptr(stream)), "rk_chem_jvp_aux")
    return out


def chem_rhs(m: Mechanism, Y, p, src=None, out=None, stream=None):
    n = _ncell(Y, m)
    out = torch.empty_like(Y) if out is None else out
    _check(_L().rk_chem_rhs(m.handle, _dptr(Y, "Y"), _dptr(src, "src", Y.numel()), float(p),
                            _dptr(out, "out", Y.numel()), n, _stream_ptr(stream)), "rk_chem_rhs")
    return out


def chem_rhs_mixed(m: Mechanism, Y, p, src=None, out=None, stream=None):
    n = _ncell(Y, m)
    out = torch.empty_like(Y) if out is None else out
    _check(_L().rk_chem_rhs_mixed(m.handle, _dptr(Y, "Y"), _dptr(src, "src", Y.numel()), float(p),
                                  _dptr(out, "out", Y.numel()), n, _stream_ptr(stream)), "rk_chem_rhs_mixed")
    return out


def chem_rhs_tc(m: Mechanism, Y, p, src=None, out=None, stream=None):
    """Source term with w = nu^T q formed on the tensor cores (rk_chem_rhs_tc)."""
    n = _ncell(Y, m)
    out = torch.empty_like(Y) if out is None else out
    _check(_L().rk_chem_rhs_tc(m.handle, _dptr(Y, "Y"), _dptr(src, "src", Y.numel()), float(p),
                               _dptr(out, "out", Y.numel()), n, _stream_ptr(stream)), "rk_chem_rhs_tc")
    return out


def chem_rhs_cv(m: Mechanism, Y, rho, src=None, out=None, stream=None):
    """Constant-volume source term (cell c at the fixed density rho[c])."""
    n = _ncell(Y, m)
    out = torch.empty_like(Y) if out is None else out
    _check(_L().rk_chem_rhs_cv(m.handle, _dptr(Y, "Y"), _dptr(src, "src", Y.numel()), _dptr(rho, "rho", n),
                               _dptr(out, "out", Y.numel()), n, _stream_ptr(stream)), "rk_chem_rhs_cv")
    return out


def chem_jvp_cv(m: Mechanism, Y, V, rho, mode=0, out=None, stream=None):
    n = _ncell(Y, m)
    out = torch.empty_like(Y) if out is None else out
    _check(_L().rk_chem_jvp_cv(m.handle, _dptr(Y, "Y"), _dptr(V, "V", Y.numel()), _dptr(rho, "rho", n),
                               _dptr(out, "out", Y.numel()), n, int(mode), _stream_ptr(stream)), "rk_chem_jvp_cv")
    return out


def chem_jvp(m: Mechanism, Y, V, p, mode=0, out=None, stream=None):
    n = _ncell(Y, m)
    out = torch.empty_like(Y) if out is None else out
    _check(_L().rk_chem_jvp(m.handle, _dptr(Y, "Y"), _dptr(V, "V", Y.numel()), float(p),
                            _dptr(out, "out", Y.numel()), n, int(mode), _stream_ptr(stream)), "rk_chem_jvp")
    return out


def rok4e_workspace_size(m: Mechanism, ncell: int, krylov_dim: int, opts: Opts | None = None) -> int:
    oc = (opts or Opts()).c()
    return int(_L().rk_rok4e_workspace_size(m.handle, int(ncell), int(krylov_dim), ctypes.byref(oc)))


def rok4e_integrate(m: Mechanism, Y, dt, rtol, atol, krylov_dim=4, *, p=101325.0, src=None, h_cell=None,
                    opts: Opts | None = None, stats=None, workspace=None, stream=None):
    """Integrate every row of Y over dt in place (rk_rok4e_integrate)."""
    n = _ncell(Y, m, _extra(opts))
    oc = (opts or Opts()).c()
    if workspace is None:
        nb = rok4e_workspace_size(m, n, krylov_dim, opts)
        workspace = torch.empty(nb, dtype=torch.uint8, device=Y.device)
    _check(_L().rk_rok4e_integrate(m.handle, _dptr(Y, "Y"), _dptr(src, "src", Y.numel()),
                                   _dptr(h_cell, "h_cell", n), n, float(p), float(dt), float(rtol), float(atol),
                                   int(krylov_dim), ctypes.byref(oc),
                                   _dptr(stats, "stats", 4 * n, torch.int32),
                                   _dptr(workspace, "workspace", dtype=torch.uint8), workspace.numel(),
                                   _stream_ptr(stream)), "rk_rok4e_integrate")
    return Y


def rkdp_integrate(m: Mechanism, Y, dt, rtol, atol, *, p=101325.0, src=None, h_cell=None,
                   opts: Opts | None = None, stats=None, workspace=None, stream=None):
    """Integrate every row of Y over dt in place with the explicit Dormand-Prince
    5(4) pair (rk_rkdp_integrate)."""
    n = _ncell(Y, m, _extra(opts))
    oc = (opts or Opts()).c()
    if workspace is None:
        workspace = torch.empty(rok4e_workspace_size(m, n, 1, opts), dtype=torch.uint8, device=Y.device)
    _check(_L().rk_rkdp_integrate(m.handle, _dptr(Y, "Y"), _dptr(src, "src", Y.numel()),
                                  _dptr(h_cell, "h_cell", n), n, float(p), float(dt), float(rtol), float(atol),
                                  ctypes.byref(oc), _dptr(stats, "stats", 4 * n, torch.int32),
                                  _dptr(workspace, "workspace", dtype=torch.uint8), workspace.numel(),
                                  _stream_ptr(stream)), "rk_rkdp_integrate")
    return Y


def simpler_split_step_workspace_size(m: Mechanism, npts: int, krylov_dim: int, opts: Opts | None = None) -> int:
    oc = (opts or Opts()).c()
    return int(_L().rk_simpler_split_step_workspace_size(m.handle, int(npts), int(krylov_dim), ctypes.byref(oc)))


def simpler_split_step(m: Mechanism, U, dt, D, dx, rtol, atol, krylov_dim=4, *, p=101325.0, h_cell=None,
                       opts: Opts | None = None, stats=None, workspace=None, stream=None):
    """One Simpler balanced split step of the 1-D reaction-diffusion system, in place."""
    n = _ncell(U, m)
    oc = (opts or Opts()).c()
    if workspace is None:
        nb = simpler_split_step_workspace_size(m, n, krylov_dim, opts)
        workspace = torch.empty(nb, dtype=torch.uint8, device=U.device)
    _check(_L().rk_simpler_split_step(m.handle, _dptr(U, "U"), _dptr(h_cell, "h_cell", n), n, float(p), float(dt),
                                      float(D), float(dx), float(rtol), float(atol), int(krylov_dim),
                                      ctypes.byref(oc), _dptr(stats, "stats", 4 * n, torch.int32),
                                      _dptr(workspace, "workspace", dtype=torch.uint8), workspace.numel(),
                                      _stream_ptr(stream)), "rk_simpler_split_step")
    return U


def simpler_split_step_ext(m: Mechanism, U, dt, rtol, atol, krylov_dim=4, *, transport=None, p=101325.0,
                           h_cell=None, opts: Opts | None = None, stats=None, workspace=None, stream=None):
    """One Simpler balanced split step with the caller's transport operator
    (rk_simpler_split_step_ext), in place.  ``transport(X, TX)`` receives two
    float64 CUDA tensors [npts, N] and writes T(X) into TX on the current
    stream; None runs the reaction step alone."""
    n = _ncell(U, m)
    N = U.shape[-1]
    oc = (opts or Opts()).c()
    if workspace is None:
        nb = int(_L().rk_split_step_workspace_size(m.handle, n, int(krylov_dim), 0, ctypes.byref(oc)))
        workspace = torch.empty(nb, dtype=torch.uint8, device=U.device)
    cb, err = ctypes.cast(None, _native.TRANSPORT_FN), []  # NULL: the reaction step alone
    if transport is not None:
        ws_lo, ws_hi = workspace.data_ptr(), workspace.data_ptr() + workspace.numel()
        nbytes = n * N * 8

        def view(ptr):  # the field at a device address the library passed: U or a workspace vector
            if ptr == U.data_ptr():
                return U.view(n, N)
            if ws_lo <= ptr and ptr + nbytes <= ws_hi:
                off = ptr - ws_lo
                return workspace[off:off + nbytes].view(torch.float64).view(n, N)
            raise RokError(f"transport callback: unknown device address {ptr:#x}")

        def trampoline(x, tx, npts, nvar, user, strm):
            try:
                transport(view(x), view(tx))
                return 0
            except Exception as e:  # re-raised after the call returns
                err.append(e)
                return 1

        cb = _native.TRANSPORT_FN(trampoline)
    rc = _L().rk_simpler_split_step_ext(m.handle, _dptr(U, "U"), _dptr(h_cell, "h_cell", n), n, float(p), float(dt),
                                        float(rtol), float(atol), int(krylov_dim), cb, None, ctypes.byref(oc),
                                        _dptr(stats, "stats", 4 * n, torch.int32),
                                        _dptr(workspace, "workspace", dtype=torch.uint8), workspace.numel(),
                                        _stream_ptr(stream))
    if err:
        raise err[0]
    _check(rc, "rk_simpler_split_step_ext")
    return U


SCHEMES = {"simpler": 0, "strang": 1, "simple_balanced": 2, "simple_balanced_transport_first": 3}


def split_step(m: Mechanism, U, dt, D, dx, rtol, atol, krylov_dim=4, scheme="simpler", *, p=101325.0,
               h_cell=None, opts: Opts | None = None, stats=None, workspace=None, stream=None):
    """One split step (any scheme of SCHEMES) of the 1-D reaction-diffusion system, in place."""
    n = _ncell(U, m)
    sc = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    oc = (opts or Opts()).c()
    if workspace is None:
        nb = int(_L().rk_split_step_workspace_size(m.handle, n, int(krylov_dim), sc, ctypes.byref(oc)))
        workspace = torch.empty(nb, dtype=torch.uint8, device=U.device)
    _check(_L().rk_split_step(m.handle, _dptr(U, "U"), _dptr(h_cell, "h_cell", n), n, float(p), float(dt),
                              float(D), float(dx), float(rtol), float(atol), int(krylov_dim), sc, ctypes.byref(oc),
                              _dptr(stats, "stats", 4 * n, torch.int32),
                              _dptr(workspace, "workspace", dtype=torch.uint8), workspace.numel(),
                              _stream_ptr(stream)), "rk_split_step")
    return U


def diffusion_1d(U, D, dx, out=None, stream=None):
    out = torch.empty_like(U) if out is None else out
    _check(_L().rk_diffusion_1d(_dptr(U, "U"), _dptr(out, "out", U.numel()), int(U.shape[0]), int(U.shape[1]),
                                float(D), float(dx), _stream_ptr(stream)), "rk_diffusion_1d")
    return out


def diffusion_1d_ghost(Uext, D, dx, out=None, stream=None):
    """D d^2U/dx^2 on the n interior rows of Uext [n + 2, nvar] (rows 0 and
    n + 1 are ghost rows): rk_diffusion_1d_ghost."""
    n = int(Uext.shape[0]) - 2
    out = torch.empty((n, Uext.shape[1]), dtype=torch.float64, device=Uext.device) if out is None else out
    _check(_L().rk_diffusion_1d_ghost(_dptr(Uext, "Uext"), _dptr(out, "out", n * Uext.shape[1]), n,
                                      int(Uext.shape[1]), float(D), float(dx), _stream_ptr(stream)),
           "rk_diffusion_1d_ghost")
    return out


def ssprk3_stage_ghost(stage, U1, Xext, S, sigma, out, D, dx, k, stream=None):
    """One SSP-RK3 stage on a slice held with ghost rows (rk_ssprk3_stage_ghost)."""
    n = int(Xext.shape[0]) - 2
    nv = int(Xext.shape[1])
    _check(_L().rk_ssprk3_stage_ghost(int(stage), _dptr(U1, "U1", n * nv), _dptr(Xext, "Xext"),
                                      _dptr(S, "S", n * nv), float(sigma), _dptr(out, "out", n * nv), n, nv,
                                      float(D), float(dx), float(k), _stream_ptr(stream)), "rk_ssprk3_stage_ghost")
    return out


class GhostTransport:
    """The library's ghost-row transport kernels: the backend of
    simpler_split_step_phases on a CUDA device."""

    def __init__(self, stream=None):
        self.stream = stream

    def diffusion(self, Xext, D, dx):
        return diffusion_1d_ghost(Xext, D, dx, stream=self.stream)

    def stage(self, stage, U1, Xext, S, sigma, out, D, dx, k):
        ssprk3_stage_ghost(stage, U1, Xext, S, sigma, out, D, dx, k, stream=self.stream)

    def empty_like(self, t):
        return torch.empty_like(t)


def simpler_split_step_phases(react, backend, Uext, dt, D, dx):
    """One Simpler balanced split step (Eq. simpler_balanced) of a slice of the
    1-D domain held with one ghost row per side (Uext [n + 2, nvar], the
    slice's points in rows 1..n, updated in place), as a generator: before
    each of the four transport evaluations it yields the array whose ghost
    rows the caller must fill (halo_exchange) -- U_n for T(U_n), then the
    state after the reaction sub-step and the two intermediate SSP-RK3 stages.
    react(U, Tn) integrates the slice's points over dt with the constant
    source Tn = T(U_n); backend supplies diffusion / stage / empty_like."""
    n = int(Uext.shape[0]) - 2
    U = Uext[1:n + 1]
    yield Uext
    Tn = backend.diffusion(Uext, D, dx)
    react(U, Tn)
    yield Uext
    V1, V2 = backend.empty_like(Uext), backend.empty_like(Uext)
    k = 0.5 * dt
    backend.stage(0, U, Uext, Tn, -1.0, V1[1:n + 1], D, dx, k)
    yield V1
    backend.stage(1, U, V1, Tn, -1.0, V2[1:n + 1], D, dx, k)
    yield V2
    backend.stage(2, U, V2, Tn, -1.0, U, D, dx, k)


def halo_exchange(ext, rank, world, group=None):
    """Fill the ghost rows of ext [n + 2, nvar] for a domain split into
    contiguous slices over ranks 0..world-1 in order: row 0 from rank - 1's
    last point, row n + 1 from rank + 1's first point (torch.distributed
    point-to-point sends and receives: NCCL for CUDA tensors, gloo on the
    CPU); at an end of the whole domain, a copy of the slice's own end point
    (zero-gradient boundary)."""
    n = int(ext.shape[0]) - 2
    ops = []
    if world > 1:
        import torch.distributed as dist

        if rank > 0:
            ops += [dist.P2POp(dist.isend, ext[1], rank - 1, group), dist.P2POp(dist.irecv, ext[0], rank - 1, group)]
        if rank < world - 1:
            ops += [dist.P2POp(dist.isend, ext[n], rank + 1, group),
                    dist.P2POp(dist.irecv, ext[n + 1], rank + 1, group)]
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
    if rank == 0:
        ext[0].copy_(ext[1])
    if rank == world - 1:
        ext[n + 1].copy_(ext[n])
    return ext


def simpler_split_step_sharded(m: Mechanism, Uext, dt, D, dx, rtol, atol, krylov_dim=4, *, rank=0, world=1,
                               group=None, p=101325.0, h_cell=None, opts: Opts | None = None, stats=None,
                               workspace=None, stream=None):
    """One Simpler split step of this rank's slice of the 1-D domain (Uext [n +
    2, nvar] with ghost rows, updated in place), exchanging one-point halos
    with the neighbouring ranks before each of the four transport evaluations.
    With every rank's slice the result is bitwise that of simpler_split_step
    on the whole domain."""
    import contextlib

    n = int(Uext.shape[0]) - 2
    if workspace is None:
        workspace = torch.empty(rok4e_workspace_size(m, n, krylov_dim, opts), dtype=torch.uint8,
                                device=Uext.device)

    def react(U, Tn):
        rok4e_integrate(m, U, dt, rtol, atol, krylov_dim, p=p, src=Tn, h_cell=h_cell, opts=opts, stats=stats,
                        workspace=workspace)

    # kernels, ghost copies and the communication all on one stream (the
    # given one made current, else the current one)
    with torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext():
        for ext in simpler_split_step_phases(react, GhostTransport(), Uext, dt, D, dx):
            halo_exchange(ext, rank, world, group)
    return Uext


def eval_exp(x, which=0, out=None, stream=None):
    """The kernels' own elementary functions on a CUDA float64 tensor (0: exp(x), 1/2: exp(+-x)
    pair; 3/4/5: the same in the mixed-precision form; 6: ln x; 7: 1/x)."""
    out = torch.empty_like(x) if out is None else out
    _check(_L().rk_eval_exp(_dptr(x, "x"), _dptr(out, "out", x.numel()), x.numel(), int(which),
                            _stream_ptr(stream)), "rk_eval_exp")
    return out


def rok4e_fixed_steps(m: Mechanism, Y, h, nsteps, krylov_dim=4, *, p=101325.0, checkpoints=None, workspace=None,
                      stream=None):
    """nsteps fixed ROK4E steps of size h in place; optionally records the state at
    the start of every step and the final state in ``checkpoints`` [nsteps+1, ncell, N]."""
    n = _ncell(Y, m)
    if workspace is None:
        workspace = torch.empty(rok4e_workspace_size(m, n, krylov_dim), dtype=torch.uint8, device=Y.device)
    _check(_L().rk_rok4e_fixed_steps(m.handle, _dptr(Y, "Y"), n, float(p), float(h), int(nsteps), int(krylov_dim),
                                     _dptr(checkpoints, "checkpoints", (int(nsteps) + 1) * Y.numel()),
                                     _dptr(workspace, "workspace", dtype=torch.uint8), workspace.numel(),
                                     _stream_ptr(stream)), "rk_rok4e_fixed_steps")
    return Y


def rok4e_adjoint_workspace_size(m: Mechanism, ncell: int, krylov_dim: int) -> int:
    return int(_L().rk_rok4e_adjoint_workspace_size(m.handle, int(ncell), int(krylov_dim)))


def rok4e_adjoint(m: Mechanism, checkpoints, ubar, h, nsteps, krylov_dim=4, *, p=101325.0, grad_u0=None,
                  workspace=None, stream=None, lanes_per_cell=0):
    """Discrete adjoint of rok4e_fixed_steps: returns (grad_lnA [Nr], grad_u0 [ncell, N] or None).
    lanes_per_cell: 4, 8, 16 or 32 lanes per cell, 0 chosen from the cell count (rk_rok4e_adjoint_ex)."""
    n = _ncell(ubar, m)
    if workspace is None:
        workspace = torch.empty(rok4e_adjoint_workspace_size(m, n, krylov_dim), dtype=torch.uint8,
                                device=ubar.device)
    grad = torch.empty(m.n_reactions, dtype=torch.float64, device=ubar.device)
    _check(_L().rk_rok4e_adjoint_ex(m.handle, _dptr(checkpoints, "checkpoints", (int(nsteps) + 1) * ubar.numel()),
                                    _dptr(ubar, "ubar"), n, float(p), float(h), int(nsteps), int(krylov_dim),
                                    int(lanes_per_cell), _dptr(grad, "grad"), _dptr(grad_u0, "grad_u0", ubar.numel()),
                                    _dptr(workspace, "workspace", dtype=torch.uint8), workspace.numel(),
                                    _stream_ptr(stream)), "rk_rok4e_adjoint_ex")
    return grad, grad_u0


class FixedStepROK4E(torch.autograd.Function):
    """u(t_end) of fixed-step ROK4E as a differentiable function of (ln A, u0).

    forward(lnA, Y0, mech, h, nsteps, M, p): lnA is a CPU float64 tensor [Nr] of
    natural logs of the pre-exponential factors (cm-mol-s, input reaction
    order; for Troe reactions the high-pressure factor), Y0 a CUDA float64
    tensor [ncell, N]; ``mech`` a synth.Mechanism supplying everything else.
    The forward pass keeps one checkpoint per step; backward runs the
    hand-written adjoint kernel (rk_rok4e_adjoint)."""

    @staticmethod
    def forward(ctx, lnA, Y0, mech, h, nsteps, M=4, p=101325.0):
        mk = mech.copy()
        mk.arrh[:, 0] = np.exp(lnA.detach().cpu().numpy())
        m = Mechanism(mk)
        Y = Y0.detach().clone().contiguous()
        ckpt = torch.empty((int(nsteps) + 1,) + tuple(Y.shape), dtype=torch.float64, device=Y.device)
        rok4e_fixed_steps(m, Y, h, nsteps, M, p=p, checkpoints=ckpt)
        ctx.m, ctx.ckpt, ctx.h, ctx.nsteps, ctx.M, ctx.p = m, ckpt, h, nsteps, M, p
        ctx.lnA_device = lnA.device
        return Y

    @staticmethod
    def backward(ctx, gY):
        g0 = torch.empty_like(gY)
        grad, g0 = rok4e_adjoint(ctx.m, ctx.ckpt, gY.contiguous(), ctx.h, ctx.nsteps, ctx.M, p=ctx.p, grad_u0=g0)
        return grad.to(ctx.lnA_device), g0, None, None, None, None, None


def probe_throughput(kind: int) -> float:
    """Measured rate (ops/s) of 0: FP64 FMA, 1: FP32 FMA, 2: FP64 exp, 3: conversions,
    4/5: FP64 FMA with 1/4 warps per SM, 6: FP64 warp instructions with one active
    lane, 7: double-float multiply-adds, 8: int -> double conversions (rk_probe_throughput)."""
    v = ctypes.c_double()
    _check(_L().rk_probe_throughput(int(kind), ctypes.byref(v)), "rk_probe_throughput")
    return v.value
