"""CPU checks of the C ABI: the library loads, exports every symbol declared in
include/rok4e.h, and validates mechanisms on the host (no GPU needed)."""

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rok4e.h")


def _lib():
    from paper_1712_00953_gb300 import _native
    from paper_1712_00953_gb300.build import build, lib_path

    if not os.path.exists(lib_path()):
        build()
    return _native.load()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rk_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_documented_calls():
    names = _declared()
    for n in ("rk_mech_load", "rk_mech_free", "rk_chem_rhs", "rk_rok4e_integrate", "rk_simpler_split_step"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = _lib()
    from paper_1712_00953_gb300.build import lib_path

    out = subprocess.run(["nm", "-D", "--defined-only", lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\s(rk_[a-z0-9_]+)$", out, flags=re.M))
    for n in _declared():
        assert n in exported, n
        assert getattr(lib, n) is not None
    from paper_1712_00953_gb300._native import SIGNATURES

    assert set(SIGNATURES) == set(_declared())


def _validate(mech):
    from paper_1712_00953_gb300._native import RkMechDesc

    lib = _lib()
    arrs = [np.ascontiguousarray(getattr(mech, k), dtype=dt) for k, dt in
            (("elem", np.int32), ("W", np.float64), ("nasa", np.float64), ("rxn_sp", np.int32),
             ("rxn_nu", np.int32), ("arrh", np.float64), ("reversible", np.uint8), ("kind", np.int32),
             ("eff", np.float64), ("falloff", np.float64))]
    d = RkMechDesc(mech.n_species, mech.n_reactions, *(a.ctypes.data for a in arrs))
    buf = ctypes.create_string_buffer(256)
    rc = lib.rk_mech_validate(ctypes.byref(d), buf, 256)
    return rc, buf.value.decode()


@pytest.mark.parametrize("name", ["small", "flame1d", "batched", "adjoint"])
def test_workload_mechanisms_validate(name):
    from synth.fields import WORKLOADS, mechanism_for

    rc, msg = _validate(mechanism_for(WORKLOADS[name]))
    assert rc == 0, msg


def _corrupt(kind):
    from synth.fields import WORKLOADS, mechanism_for

    m = mechanism_for(WORKLOADS["flame1d"]).copy()
    if kind == "imbalance":
        j = int(np.where(m.rxn_sp[:, 3] >= 0)[0][0])
        m.rxn_sp[j, 3] = (m.rxn_sp[j, 3] + 1) % m.n_species
    elif kind == "index":
        m.rxn_sp[0, 0] = m.n_species
    elif kind == "sign":
        m.rxn_nu[0, 0] = -m.rxn_nu[0, 0]
    elif kind == "three":
        j = int(np.where((m.rxn_sp[:, 1] >= 0) & (m.rxn_nu[:, 0] == -1))[0][0])
        m.rxn_nu[j, 0] = -2
    elif kind == "A":
        m.arrh[3, 0] = 0.0
    elif kind == "kind":
        m.kind[2] = 7
    elif kind == "nasa":
        m.nasa[1, 10] += 0.5
    elif kind == "W":
        m.W[0] = -1.0
    elif kind == "troe":
        j = int(np.where(m.kind == 2)[0][0])
        m.falloff[j, 4] = 0.0
    return m


@pytest.mark.parametrize("kind,needle", [("imbalance", "not balanced"), ("index", "out of range"),
                                         ("sign", "nu"), ("three", "two molecules"), ("A", "A > 0"),
                                         ("kind", "kind"), ("nasa", "discontinuous"), ("W", "molar mass"),
                                         ("troe", "Troe")])
def test_invalid_mechanisms_are_rejected(kind, needle):
    rc, msg = _validate(_corrupt(kind))
    assert rc == -2
    assert needle in msg, msg


def test_status_strings():
    lib = _lib()
    assert lib.rk_status_string(0) == b"ok"
    assert lib.rk_status_string(-2) == b"mechanism invalid"
    assert lib.rk_status_string(-99) == b"unknown status"


def test_null_arguments_rejected_without_gpu():
    lib = _lib()
    assert lib.rk_mech_validate(None, None, 0) == -2
    assert lib.rk_mech_free(None) == 0
    assert lib.rk_chem_rhs(None, None, None, 1.0, None, 1, None) == -1
    assert lib.rk_rok4e_integrate(None, None, None, None, 1, 1.0, 1.0, 1.0, 1.0, 4, None, None, None, 0, None) == -1
    assert lib.rk_diffusion_1d(None, None, 4, 3, 1.0, 1.0, None) == -1
