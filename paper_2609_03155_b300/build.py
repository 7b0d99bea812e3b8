"""Build libdpg.so in-tree with nvcc for sm_103a (B300).

The library is a plain C ABI (include/dpg.h) over CUDA kernels and host C++
setup code; Python reaches it through ctypes (``_lib.py``).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SOURCES = ["tables.cpp", "setup.cpp", "element.cu", "quad_sf.cu", "factor_tc.cu", "quad_tc.cu", "solve.cu", "adjoint.cu", "power.cu", "abi.cu"]
LIB = os.path.join(HERE, "libdpg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    raise RuntimeError("nvcc not found")


def build(verbose=False, extra=()):
    """Compile every source of the library into paper_2609_03155_b300/libdpg.so."""
    src = [os.path.join(HERE, "csrc", f) for f in SOURCES]
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-shared",
           "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-x", "cu", *src, "-o", LIB, *extra]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
