"""Build libmfsolve.so in-tree with nvcc for sm_103a (B300).

    python -m paper_2306_08994_b300.build [--verbose] [--force]

The library is the C ABI declared in include/mfsolve.h; the Python binding
loads it from this folder.  Each source is compiled to an object under
_build/ (in parallel; a source is recompiled when it, a shared header or the
public header is newer than its object) and the objects are linked into the
shared library.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmfsolve.so")
OBJ = os.path.join(ROOT, "_build")
SOURCES = ["analysis.cpp", "analysis_csr.cpp", "capi.cpp", "executor.cu", "noalloc.cu", "autotune.cpp"]
HEADERS = ["mf_internal.h", "kernels_factor.cuh", "kernels_foata.cuh", "kernels_solve.cuh", "kernels_subtree.cuh",
           "kernels_tc.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _headers_mtime() -> float:
    deps = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "mfsolve.h")]
    return max(os.path.getmtime(d) for d in deps if os.path.exists(d))


def _obj(src: str) -> str:
    return os.path.join(OBJ, src + ".o")


def _stale_sources(force: bool):
    hm = _headers_mtime()
    out = []
    for s in SOURCES:
        o = _obj(s)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(hm, os.path.getmtime(os.path.join(CSRC, s))):
            out.append(s)
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    os.makedirs(OBJ, exist_ok=True)
    todo = _stale_sources(force)
    if not todo and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(_obj(s)) for s in SOURCES):
        return LIB
    base = [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
            "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if verbose:
        base += ["-Xptxas", "-v"]

    def compile_one(src):
        o = _obj(src)
        subprocess.check_call(base + ["-c", os.path.join(CSRC, src), "-o", o + ".tmp"])
        os.replace(o + ".tmp", o)

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for f in [ex.submit(compile_one, s) for s in todo]:
            f.result()
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", LIB + ".tmp"] + [_obj(s) for s in SOURCES])
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="--verbose" in sys.argv)
    print(LIB)
