"""Build libperch.so in-tree with nvcc for sm_103a (no torch extension machinery).

The library exposes only the C ABI of include/perch.h, so it is compiled as a
plain shared object: each .cu file is compiled in parallel to an object file,
then linked with the static CUDA runtime.  Every translation unit uses
-fmad=false: the scoring path's integer decisions (snapping, depth, distances)
depend on uncontracted single-precision operations.
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libperch.so")
BUILD_DIR = os.path.join(PKG, "_build")
# debug build: every scorer index checked before use (PERCH_CHECKS), violations
# reported through the device error word; same ABI, slower
LIB_CHECKS = os.path.join(PKG, "libperch_checks.so")
BUILD_DIR_CHECKS = os.path.join(PKG, "_build_checks")
SOURCES = ["perch_api.cu", "perch_batch.cu", "perch_serve.cu", "perch_refine.cu", "perch_tree.cu", "perch_kernels.cu",
           "perch_noalloc.cu", "perch_microbench.cu", "perch_metrics.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-prec-div=true", "-prec-sqrt=true",
              "-Xcompiler", "-fPIC,-fvisibility=hidden", "--expt-relaxed-constexpr"]


def _nvcc():
    for cand in (os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc"), "nvcc"):
        if os.path.sep not in cand or os.path.exists(cand):
            return cand
    return "nvcc"


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    files.append(os.path.abspath(__file__))
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra_flags=(), checks: bool = False) -> str:
    """Compile the CUDA sources and link libperch.so (checks=True: the debug
    library libperch_checks.so, with -DPERCH_CHECKS); returns its path."""
    lib = LIB_CHECKS if checks else LIB
    build_dir = BUILD_DIR_CHECKS if checks else BUILD_DIR
    if checks:
        extra_flags = (*extra_flags, "-DPERCH_CHECKS=1")
    if not force and up_to_date(lib):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra_flags, "-I", INCLUDE, "-I", CSRC, "-c",
               os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(cmd[-3])
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    tmp = lib + ".tmp"
    link = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp]
    if verbose:
        print(" ".join(link), flush=True)
    subprocess.check_call(link)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, checks="--checks" in sys.argv)
