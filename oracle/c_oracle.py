"""The C oracle (oracle/c/rok4e_oracle.c) through ctypes -- TEST INFRASTRUCTURE.

A compiled restatement of the same method as the numpy oracle (kinetics,
ROK4E with dense Arnoldi, Simpler split steps), used where the numpy oracle
is too slow: split-step horizons of 1000 steps and the timed CPU baseline on
every host core.  It shares no code with the CUDA library.  It is pinned
against the numpy oracle in tests/test_oracle_c.py.

    build()                       compile oracle/c/_lib/liboracle_rok4e.so (gcc -O3 -fopenmp)
    COracle(mech)                 a mechanism (synth.Mechanism) loaded into it
    .rhs(u, p, src) / .jvp(u, v, p, mode)
    .integrate(U, dt, rtol, atol, M, src=, h0=, replay=, jv_mode=, threads=) -> (U_out, h_last, stats)
    .simpler_steps(U, h, nsteps, dt, D, dx, rtol, atol, M, replay=, threads=) -> (U_out, h, stats)
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "c", "rok4e_oracle.c")
LIB = os.path.join(HERE, "c", "_lib", "liboracle_rok4e.so")
_LIB = None
P = ctypes.c_void_p


def build(verbose=False) -> str:
    """Compile the C oracle in-tree (plain C99, -O3, OpenMP; no -march flags, no
    fused multiply-add contraction, so x86 and Arm builds round alike)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".tmp"
    cmd = ["gcc", "-O3", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError(f"C oracle build failed: {' '.join(cmd)}\n{r.stdout.decode(errors='replace')}")
    if verbose and r.stdout.strip():
        print(r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB):
            build()
        lib = ctypes.CDLL(LIB)
        lib.orc_mech_new.restype = P
        lib.orc_mech_new.argtypes = [ctypes.c_int, ctypes.c_int] + [P] * 9
        lib.orc_mech_free.argtypes = [P]
        lib.orc_rhs.argtypes = [P, P, P, ctypes.c_double, P]
        lib.orc_jvp.argtypes = [P, P, P, ctypes.c_double, ctypes.c_int, P]
        lib.orc_integrate.argtypes = [P, P, P, P, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P, ctypes.c_int]
        lib.orc_simpler_steps.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, P, P, ctypes.c_int, P, ctypes.c_int]
        _LIB = lib
    return _LIB


def _p(a):
    return None if a is None else a.ctypes.data_as(P)


class COracle:
    def __init__(self, mech):
        lib = _lib()
        self._keep = [np.ascontiguousarray(mech.W, dtype=np.float64),
                      np.ascontiguousarray(mech.nasa, dtype=np.float64),
                      np.ascontiguousarray(mech.rxn_sp, dtype=np.int32),
                      np.ascontiguousarray(mech.rxn_nu, dtype=np.int32),
                      np.ascontiguousarray(mech.arrh, dtype=np.float64),
                      np.ascontiguousarray(mech.reversible, dtype=np.uint8),
                      np.ascontiguousarray(mech.kind, dtype=np.int32),
                      np.ascontiguousarray(mech.eff, dtype=np.float64),
                      np.ascontiguousarray(mech.falloff, dtype=np.float64)]
        self.ns, self.nr = int(mech.W.shape[0]), int(mech.arrh.shape[0])
        self.h = lib.orc_mech_new(self.ns, self.nr, *(_p(a) for a in self._keep))
        if not self.h:
            raise ValueError("mechanism outside the C oracle's limits")

    def __del__(self):
        try:
            _lib().orc_mech_free(self.h)
        except Exception:
            pass

    def rhs(self, u, p, src=None):
        u = np.ascontiguousarray(u, dtype=np.float64)
        s = None if src is None else np.ascontiguousarray(src, dtype=np.float64)
        f = np.empty_like(u)
        _lib().orc_rhs(self.h, _p(u), _p(s), float(p), _p(f))
        return f

    def jvp(self, u, v, p, mode=0):
        u = np.ascontiguousarray(u, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.empty_like(u)
        _lib().orc_jvp(self.h, _p(u), _p(v), float(p), int(mode), _p(out))
        return out

    def integrate(self, U, dt, rtol, atol, M, *, p=101325.0, src=None, h0=None, replay=None, jv_mode=0,
                  record_cap=0, threads=None):
        """Every row of U over dt (copies; returns (U_out, h_last, stats [n, 4]),
        plus the recorded attempts [n, record_cap] when record_cap > 0).
        replay: [n, cap] signed steps (+h accepted, -h rejected, 0 ends)."""
        U = np.array(U, dtype=np.float64, order="C")
        n = U.shape[0]
        s = None if src is None else np.ascontiguousarray(src, dtype=np.float64)
        h = np.zeros(n) if h0 is None else np.array(np.broadcast_to(h0, (n,)), dtype=np.float64)
        rp = None if replay is None else np.ascontiguousarray(replay, dtype=np.float64)
        cap = 0 if rp is None else rp.shape[1]
        rec = None
        if record_cap > 0:
            if rp is not None and record_cap != cap:
                raise ValueError("record_cap must equal the replay's cap")
            cap = record_cap
            rec = np.zeros((n, cap))
        st = np.zeros((n, 4), dtype=np.int32)
        rc = _lib().orc_integrate(self.h, _p(U), _p(s), _p(h), n, float(p), float(dt), float(rtol), float(atol),
                                  int(M), int(jv_mode), _p(rp), _p(rec), cap, _p(st),
                                  threads or (os.cpu_count() or 1))
        if rc:
            raise ValueError("orc_integrate: bad arguments")
        return (U, h, st) if rec is None else (U, h, st, rec)

    def simpler_steps(self, U, h, nsteps, dt, D, dx, rtol, atol, M, *, p=101325.0, replay=None, record_cap=0,
                      threads=None):
        """nsteps Simpler split steps of the 1-D system (copies; returns (U, h, stats [nsteps, npts, 4]),
        plus the recorded attempts [nsteps, npts, record_cap] when record_cap > 0).
        replay: [nsteps, npts, cap] or None."""
        U = np.array(U, dtype=np.float64, order="C")
        h = np.array(h, dtype=np.float64)
        npts = U.shape[0]
        rp = None if replay is None else np.ascontiguousarray(replay, dtype=np.float64)
        cap = 0 if rp is None else rp.shape[2]
        rec = None
        if record_cap > 0:
            if rp is not None and record_cap != cap:
                raise ValueError("record_cap must equal the replay's cap")
            cap = record_cap
            rec = np.zeros((nsteps, npts, cap))
        st = np.zeros((nsteps, npts, 4), dtype=np.int32)
        rc = _lib().orc_simpler_steps(self.h, _p(U), _p(h), npts, float(p), float(dt), float(D), float(dx),
                                      float(rtol), float(atol), int(M), int(nsteps), _p(rp), _p(rec), cap, _p(st),
                                      threads or (os.cpu_count() or 1))
        if rc:
            raise ValueError("orc_simpler_steps: bad arguments")
        return (U, h, st) if rec is None else (U, h, st, rec)
