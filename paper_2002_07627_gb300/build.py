"""Build the CUDA library libimf.so in-tree for sm_103a (nvcc, one -gencode, parallel TUs).

Output: paper_2002_07627_gb300/_build/libimf.so (git-ignored). Also builds
_build/libimf_hosttest.so, a host-only library that runs the FFT building blocks of the
kernels on the CPU for the host-side unit tests.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libimf.so")
HOSTLIB = os.path.join(BUILD, "libimf_hosttest.so")

CUDA_SOURCES = ["imf_api.cu", "fft_kernels.cu", "fft2_kernels.cu", "fft_tma.cu", "fft_tma_x.cu", "imf_kernels.cu",
                "erode.cu", "direct_tc.cu", "noalloc.cu", "topopt2d.cu"]
# sources compiled more than once with different defines: (source, object name, defines); the
# six instances of the TMA-fed axis pass build in parallel
CUDA_VARIANTS = [("fft_tma_inst.cu", f"fft_tma_{'b' if big else 's'}{v}.o", [f"-DIMF_TMA_BIG={big}", f"-DIMF_TMA_VARIANT={v}"])
                 for big in (0, 1) for v in (0, 1, 2)]
HOST_TEST_SOURCES = ["hosttest.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libimf")


def _deps():
    out = []
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cuh", ".h")):
                out.append(os.path.join(d, f))
    return out


def _stale(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(p) > t for p in _deps() + [__file__])


def _flags():
    return ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
            "-I", INCLUDE, "-I", CSRC]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA translation unit in parallel and link libimf.so."""
    os.makedirs(BUILD, exist_ok=True)
    if force or _stale(LIB):
        cc = nvcc()
        objs, procs = [], []
        units = [(s, s.replace(".cu", ".o"), []) for s in CUDA_SOURCES] + CUDA_VARIANTS
        for src, oname, defs in units:
            obj = os.path.join(BUILD, oname)
            cmd = [cc, *ARCH, *_flags(), *defs, "-c", os.path.join(CSRC, src), "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), src))
            objs.append(obj)
        errs = []
        for p, src in procs:
            out, _ = p.communicate()
            if p.returncode != 0:
                errs.append(f"--- {src}\n{out.decode(errors='replace')}")
            elif verbose and out:
                print(out.decode(errors="replace"), file=sys.stderr)
        if errs:
            raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=BUILD)
        os.close(fd)
        subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"],
                       check=True)
        os.replace(tmp, LIB)
    if force or _stale(HOSTLIB):
        cc = nvcc()
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=BUILD)
        os.close(fd)
        cmd = [cc, *ARCH, *_flags(), "-shared", "-o", tmp] + [os.path.join(CSRC, s) for s in HOST_TEST_SOURCES]
        subprocess.run(cmd, check=True, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        os.replace(tmp, HOSTLIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
