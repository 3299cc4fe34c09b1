"""Build the CUDA library ``libcgdem.so`` in-tree for sm_103a with nvcc."""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libcgdem.so")
LIB_CHECKED = os.path.join(BUILD, "libcgdem_checked.so")   # -DDEM_CHECKS=1: in-kernel bounds checks

SOURCES = ["dem.cu", "dem_noalloc.cu", "dem_coupling.cu"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checks: bool = False) -> str:
    """Compile every .cu under csrc/ to an object, then link the shared library.  checks: the
    bounds-checked variant (the step kernel's gathered indices and the list build's cell codes
    and candidate ranges tested in the kernels; a violation is reported as DEM_ERR_BOUNDS), built
    beside the plain one."""
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "dem.h"))
    objs = []
    jobs = []
    tag = "_checked" if checks else ""
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", tag + ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([_nvcc()] + NVCC_FLAGS + (["-DDEM_CHECKS=1"] if checks else []) + ["-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)

    with ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        list(ex.map(run, jobs))
    lib = LIB_CHECKED if checks else LIB
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        run([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp] + objs)
        os.replace(tmp, lib)
    return lib


def build_all(force: bool = False, verbose: bool = False) -> tuple[str, str]:
    """The plain library and the bounds-checked one, compiled side by side."""
    with ThreadPoolExecutor(max_workers=2) as ex:
        plain = ex.submit(build, force, verbose, False)
        checked = ex.submit(build, force, verbose, True)
        return plain.result(), checked.result()


if __name__ == "__main__":
    import sys
    print(build(verbose=True, checks="--checks" in sys.argv))
