"""ctypes declarations of the C ABI in include/rok4e.h (argument marshalling only)."""

from __future__ import annotations

import ctypes
import os

from .build import lib_path

# rk_transport_fn: int (*)(const double* U, double* TU, int64_t npts, int32_t nvar, void* user, void* stream)
TRANSPORT_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                ctypes.c_void_p, ctypes.c_void_p)

c_double_p = ctypes.POINTER(ctypes.c_double)
c_int32_p = ctypes.POINTER(ctypes.c_int32)


class RkMechDesc(ctypes.Structure):
    _fields_ = [
        ("n_species", ctypes.c_int32),
        ("n_reactions", ctypes.c_int32),
        ("elem", ctypes.c_void_p),
        ("W", ctypes.c_void_p),
        ("nasa", ctypes.c_void_p),
        ("rxn_sp", ctypes.c_void_p),
        ("rxn_nu", ctypes.c_void_p),
        ("arrh", ctypes.c_void_p),
        ("reversible", ctypes.c_void_p),
        ("kind", ctypes.c_void_p),
        ("eff", ctypes.c_void_p),
        ("falloff", ctypes.c_void_p),
    ]


class RkOpts(ctypes.Structure):
    _fields_ = [
        ("jv_mode", ctypes.c_int32),
        ("max_attempts", ctypes.c_int32),
        ("lanes_per_cell", ctypes.c_int32),
        ("cells_per_block", ctypes.c_int32),
        ("h0", ctypes.c_double),
        ("fixed_h", ctypes.c_double),
        ("trace_cap", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("trace", ctypes.c_void_p),
        ("ev_begin", ctypes.c_void_p),
        ("ev_end", ctypes.c_void_p),
        ("queue_order", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32),
        ("reactor", ctypes.c_int32),
        ("reserved1", ctypes.c_int32),
        ("rho_cell", ctypes.c_void_p),
    ]


# name -> (restype, argtypes)
SIGNATURES = {
    "rk_mech_validate": (ctypes.c_int, [ctypes.POINTER(RkMechDesc), ctypes.c_char_p, ctypes.c_size_t]),
    "rk_mech_load": (ctypes.c_int, [ctypes.POINTER(RkMechDesc), ctypes.POINTER(ctypes.c_void_p)]),
    "rk_mech_free": (ctypes.c_int, [ctypes.c_void_p]),
    "rk_mech_info": (ctypes.c_int, [ctypes.c_void_p, c_int32_p, c_int32_p, ctypes.POINTER(ctypes.c_size_t)]),
    "rk_chem_rhs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                   ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "rk_chem_jvp": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                   ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p]),
    "rk_chem_rhs_mixed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                         ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "rk_chem_rhs_tc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                      ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "rk_chem_rhs_cv": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "rk_chem_jvp_cv": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p]),
    "rk_chem_rhs_aux": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_void_p]),
    "rk_chem_jvp_aux": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p]),
    "rk_rok4e_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                                  ctypes.POINTER(RkOpts)]),
    "rk_rok4e_integrate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int32, ctypes.POINTER(RkOpts),
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "rk_rkdp_integrate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.POINTER(RkOpts),
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "rk_simpler_split_step_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                                               ctypes.POINTER(RkOpts)]),
    "rk_simpler_split_step_ext": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                 ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_int32, TRANSPORT_FN, ctypes.c_void_p,
                                                 ctypes.POINTER(RkOpts), ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_size_t, ctypes.c_void_p]),
    "rk_simpler_split_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                             ctypes.POINTER(RkOpts), ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_size_t, ctypes.c_void_p]),
    "rk_simpler_split_step_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                     ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                                     ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                     ctypes.c_double, ctypes.c_int32, ctypes.POINTER(RkOpts),
                                                     ctypes.c_void_p, ctypes.c_void_p]),
    "rk_split_step_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                                       ctypes.c_int32, ctypes.POINTER(RkOpts)]),
    "rk_split_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.POINTER(RkOpts), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                     ctypes.c_void_p]),
    "rk_rok4e_fixed_steps": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "rk_rok4e_adjoint_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32]),
    "rk_rok4e_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                        ctypes.c_void_p]),
    "rk_rok4e_adjoint_ex": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_size_t, ctypes.c_void_p]),
    "rk_diffusion_1d": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_void_p]),
    "rk_diffusion_1d_ghost": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_void_p]),
    "rk_ssprk3_stage_ghost": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_double, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_void_p]),
    "rk_probe_throughput": (ctypes.c_int, [ctypes.c_int32, c_double_p]),
    "rk_eval_exp": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                   ctypes.c_void_p]),
    "rk_status_string": (ctypes.c_char_p, [ctypes.c_int32]),
    "rk_last_error": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_size_t]),
}

_LIB = None


def load(path: str | None = None):
    """Load librok4e.so (raises if it has not been built: there is no fallback)."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or lib_path()
    if not os.path.exists(p):
        raise ImportError(f"{p} not found: build it with `python -m paper_1712_00953_gb300.build` "
                          "(the library has no CPU fallback)")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _LIB = lib
    return lib


def last_error(lib) -> str:
    buf = ctypes.create_string_buffer(512)
    lib.rk_last_error(buf, 512)
    return buf.value.decode(errors="replace")
