"""Build libmfsolve.so in-tree with nvcc for sm_103a (B300).

    python -m paper_2306_08994_b300.build [--verbose]

The library is the C ABI declared in include/mfsolve.h; the Python binding
loads it from this folder.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmfsolve.so")
SOURCES = ["analysis.cpp", "capi.cpp", "executor.cu", "noalloc.cu", "autotune.cpp"]
HEADERS = ["mf_internal.h", "kernels_factor.cuh", "kernels_solve.cuh", "kernels_subtree.cuh", "kernels_tc.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "mfsolve.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    cmd = [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    cmd += [os.path.join(CSRC, s) for s in SOURCES] + ["-o", LIB + ".tmp"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="--verbose" in sys.argv)
    print(LIB)
