"""Build libhotrg.so (sm_103a) in-tree with nvcc.

Each ``csrc/*.cu`` translation unit is compiled in parallel to an object file
under ``_build/`` and linked into ``paper_2602_05900_gb300/libhotrg.so``
against the shared CUDA runtime.  Nothing is installed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libhotrg.so")
LIB_CHECKED = os.path.join(HERE, "libhotrg_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.isdir(home):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _needs(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra_flags=None, checked: bool = False) -> str:
    """Compile every CUDA source and link the shared library; returns its path.

    checked=True builds the bounds-checked variant (-DHOTRG_CHECKED=1: every
    mapped access of the GEMM, gather and epilogue kernels is compared with its
    buffer, a bad one is skipped and reported as HOTRG_EBOUNDS) as
    libhotrg_checked.so, with its own object files."""
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    build_dir = BUILD + ("_checked" if checked else "")
    lib = LIB_CHECKED if checked else LIB
    os.makedirs(build_dir, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(ROOT, "include", "hotrg.h")]
    flags = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
             "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")] + ARCH
    flags += list(extra_flags or [])
    if checked:
        flags += ["-DHOTRG_CHECKED=1"]
    if os.environ.get("HOTRG_PTXAS_VERBOSE"):
        flags += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
        if _needs(obj, [src] + headers + [__file__]):
            cmd = [nvcc] + flags + ["-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd), flush=True)
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
            if r.stderr.strip() and (verbose or os.environ.get("HOTRG_PTXAS_VERBOSE")):
                print(r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(sources))) as ex:
        objs = list(ex.map(compile_one, sources))
    if _needs(lib, objs):
        libdir = os.path.join(cuda, "lib64")
        if not os.path.isdir(libdir):
            libdir = os.path.join(cuda, "lib")
        cmd = [nvcc, "-shared", "-cudart", "shared"] + ARCH + ["-o", lib] + objs + [
            "-L", libdir, "-Xlinker", "-rpath", "-Xlinker", libdir]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
