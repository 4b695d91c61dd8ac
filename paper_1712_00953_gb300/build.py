"""Build the C-ABI shared library librok4e.so in-tree (nvcc + g++, sm_103a).

    python -m paper_1712_00953_gb300.build

Two translation units compile in parallel: the host-only mechanism packing
(g++) and the kernels plus C ABI (nvcc, -gencode arch=compute_103a,code=sm_103a).
The CUDA runtime is linked statically so the library only needs the driver.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB_NAME = "librok4e.so"
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librok4e.so")


def lib_path() -> str:
    return os.path.join(OUT_DIR, LIB_NAME)


def build(verbose: bool = False, extra_nvcc=()) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    bdir = os.path.join(OUT_DIR, "obj")
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    cu = os.path.join(CSRC, "rok4e_kernels.cu")
    cpp = os.path.join(CSRC, "mech.cpp")
    o_cu = os.path.join(bdir, "rok4e_kernels.o")
    o_cpp = os.path.join(bdir, "mech.o")
    cmd_cu = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
              "--expt-relaxed-constexpr", "-c", cu, "-o", o_cu, *extra_nvcc]
    cmd_cpp = ["g++", "-O2", "-std=c++17", "-fPIC", "-I", INCLUDE, "-I", CSRC, "-c", cpp, "-o", o_cpp]
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for c in (cmd_cu, cmd_cpp)]
    outs = [p.communicate()[0].decode(errors="replace") for p in procs]
    for c, p, o in zip((cmd_cu, cmd_cpp), procs, outs):
        if verbose and o.strip():
            print(o)
        if p.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(c)}\n{o}")
    tmp = lib_path() + ".tmp"
    cmd_ld = [nvcc, ARCH, "-shared", "-cudart", "static", o_cu, o_cpp, "-o", tmp]
    r = subprocess.run(cmd_ld, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd_ld)}\n{r.stdout.decode(errors='replace')}")
    os.replace(tmp, lib_path())
    return lib_path()


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
