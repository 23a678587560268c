"""Build libamgf.so in place: host setup (g++ -fopenmp) + sm_103a CUDA (nvcc), linked with nvcc.

Only one architecture is generated: ``-gencode arch=compute_103a,code=sm_103a``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libamgf.so")
SOURCES = ["setup.cpp", "amgf.cu"]
HEADERS = ["setup.h", "kernels.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libamgf.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INC, "amgf.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    tmp = tempfile.mkdtemp(prefix="amgf_build_", dir=HERE)
    try:
        o_setup = os.path.join(tmp, "setup.o")
        o_cuda = os.path.join(tmp, "amgf.o")
        cmds = [
            ["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-ffp-contract=off", "-I", INC,
             "-c", os.path.join(CSRC, "setup.cpp"), "-o", o_setup],
            [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-I", INC, "-Xcompiler", "-fPIC,-fopenmp",
             "-Xptxas", "-v" if verbose else "-O3",
             "-c", os.path.join(CSRC, "amgf.cu"), "-o", o_cuda],
        ]
        procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
        for c, p in zip(cmds, procs):
            out, _ = p.communicate()
            if verbose and out:
                print(out)
            if p.returncode != 0:
                raise RuntimeError(f"build failed: {' '.join(c)}\n{out}")
        so_tmp = os.path.join(tmp, "libamgf.so")
        link = [nvcc, *ARCH, "-shared", "-o", so_tmp, o_setup, o_cuda, "-Xcompiler", "-fopenmp", "-lgomp"]
        r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(link)}\n{r.stdout}")
        os.replace(so_tmp, LIB)
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
