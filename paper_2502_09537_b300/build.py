"""Build ``libkgs.so`` (the C-ABI library of ``include/kgs.h``) for sm_103a.

The library is built in-tree next to this file with plain nvcc, so the binary
travels with the repository checkout.  ``python -m paper_2502_09537_b300.build``
rebuilds it; ``build(verbose=True)`` also prints ptxas register/spill reports.
"""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libkgs.so")
# the same sources with every index check of KGS_DEBUG_BOUNDS compiled in
LIB_DEBUG = os.path.join(HERE, "libkgs_debug.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    deps += glob.glob(os.path.join(ROOT, "include", "*.h"))
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug_bounds: bool = False) -> str:
    """Build libkgs.so, or with debug_bounds the index-checking libkgs_debug.so."""
    lib = LIB_DEBUG if debug_bounds else LIB
    if not force and not _stale(lib):
        return lib
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
           "-shared", "-cudart", "shared", "-I", os.path.join(ROOT, "include"),
           "-Xlinker", "-rpath=/usr/local/cuda/lib64", "-o", lib + ".tmp", *sources()]
    if debug_bounds:
        cmd.insert(1, "-DKGS_DEBUG_BOUNDS")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                debug_bounds="--debug-bounds" in sys.argv))
