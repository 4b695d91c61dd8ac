"""Build the C-ABI shared library librok4e.so in-tree (nvcc + g++, sm_103a).

    python -m paper_1712_00953_gb300.build

The translation units compile in parallel: the host-only mechanism packing
(g++), the C ABI with the small kernels (rok4e_kernels.cu) and one file per
group of heavy kernel instantiations (k_*.cu), all with nvcc -gencode
arch=compute_103a,code=sm_103a.  The CUDA runtime is linked statically so the
library only needs the driver.
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
    cus = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cmds, objs = [], []
    for f in cus:
        o = os.path.join(bdir, f[:-3] + ".o")
        cmds.append([nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                     "--expt-relaxed-constexpr", "-c", os.path.join(CSRC, f), "-o", o, *extra_nvcc])
        objs.append(o)
    o_cpp = os.path.join(bdir, "mech.o")
    cmds.append(["g++", "-O2", "-std=c++17", "-fPIC", "-I", INCLUDE, "-I", CSRC, "-c", os.path.join(CSRC, "mech.cpp"),
                 "-o", o_cpp])
    objs.append(o_cpp)
    # at most one compile per core
    jobs = max(1, min(len(cmds), os.cpu_count() or 1))
    pending, running = list(cmds), []
    while pending or running:
        while pending and len(running) < jobs:
            c = pending.pop(0)
            running.append((c, subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        c, p = running.pop(0)
        o = p.communicate()[0].decode(errors="replace")
        if verbose and o.strip():
            print(o)
        if p.returncode != 0:
            for _, q in running:
                q.wait()
            raise RuntimeError(f"compile failed: {' '.join(c)}\n{o}")
    tmp = lib_path() + ".tmp"
    cmd_ld = [nvcc, ARCH, "-shared", "-cudart", "static", *objs, "-o", tmp]
    r = subprocess.run(cmd_ld, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd_ld)}\n{r.stdout.decode(errors='replace')}")
    os.replace(tmp, lib_path())
    return lib_path()


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
