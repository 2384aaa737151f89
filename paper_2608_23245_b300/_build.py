"""Build libfdx.so in-tree with nvcc for sm_103a (B300).

`build(debug=True)` writes libfdx_debug.so instead: the same sources with
FDX_DEBUG defined (device-side bounds checks that record violations for
fdx_debug_status) and relocatable device code, so that the kernels of all
files share one status word.  Tests load it in a process of its own."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "libfdx.so")
LIB_DEBUG = os.path.join(PKG, "libfdx_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(PKG, "csrc", "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(PKG, "csrc", "*.cuh")) + [os.path.join(ROOT, "include", "fdx.h")])


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in sources() + headers())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    if not force and not stale(lib):
        return lib
    nvcc = os.environ.get("NVCC", "nvcc")
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(PKG, "csrc"),
           "-o", lib + ".tmp", *sources()]
    if debug:
        cmd[1:1] = ["-DFDX_DEBUG", "-rdc=true"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv, debug="--debug" in sys.argv)
    print(LIB_DEBUG if "--debug" in sys.argv else LIB)
