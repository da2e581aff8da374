"""Builds the CUDA library libcbspmv.so in-tree (paper_2605_18515_gb300/_build/).

nvcc compiles the device code for sm_103a only; the host analyser is plain C++17. The
translation units compile in parallel and the result links against the static CUDA
runtime, so the library has no dependency on PyTorch.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(BUILD, "libcbspmv.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
              "--expt-relaxed-constexpr", "-I" + INCLUDE]
CXX_FLAGS = ["-O3", "-std=c++17", "-fPIC", "-pthread", "-I" + INCLUDE]

SOURCES_CU = ["kernels.cu", "capi.cu", "noalloc.cu", "serve.cu", "measure.cu", "spmm.cu", "analyze_dev.cu"]
SOURCES_CXX = ["analyze.cpp"]
_lock = threading.Lock()


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return cand


def _inputs() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libcbspmv.so; returns its path. Raises on compiler errors."""
    with _lock:
        if not force and up_to_date():
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        nvcc = _nvcc()
        cxx = shutil.which("g++") or "g++"
        jobs = []
        objs = []
        for f in SOURCES_CU:
            o = os.path.join(BUILD, f + ".o")
            objs.append(o)
            jobs.append([nvcc, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, f), "-o", o])
        for f in SOURCES_CXX:
            o = os.path.join(BUILD, f + ".o")
            objs.append(o)
            jobs.append([cxx, *CXX_FLAGS, "-c", os.path.join(CSRC, f), "-o", o])
        procs = [subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for j in jobs]
        errors = []
        for j, p in zip(jobs, procs):
            out, _ = p.communicate()
            if verbose and out:
                sys.stdout.write(out.decode(errors="replace"))
            if p.returncode != 0:
                errors.append(" ".join(j) + "\n" + out.decode(errors="replace"))
        if errors:
            raise RuntimeError("CUDA library build failed:\n" + "\n".join(errors))
        tmp = LIB + f".{os.getpid()}.tmp"
        link = [nvcc, *ARCH, "-shared", "-cudart", "static", "-Xcompiler", "-pthread", "-o", tmp, *objs]
        r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + " ".join(link) + "\n" + r.stdout.decode(errors="replace"))
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
