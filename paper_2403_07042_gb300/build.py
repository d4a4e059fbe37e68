"""Builds libqed.so in-tree with nvcc for sm_103a (one -gencode, objects in parallel)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libqed.so")
# the debug build with device bounds checks (QED_CHECKS=1): its own objects and library
BUILD_CHECKS = os.path.join(HERE, "_build_checks")
LIB_CHECKS = os.path.join(HERE, "libqed_checks.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["builder.cpp", "capi.cu", "kernels_f64.cu", "split.cu", "gemm_tc.cu", "gemm_static.cu", "expm.cu", "adjoint.cu"]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libqed")
    return path


def _flags(src, checks=False):
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if checks:
        common += ["-DQED_CHECKS=1"]
    if src.endswith(".cpp"):
        return ["-x", "c++"] + common
    return ARCH + ["-lineinfo", "--expt-relaxed-constexpr"] + common


def _compile(src, verbose, checks=False):
    obj = os.path.join(BUILD_CHECKS if checks else BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + _flags(src, checks)
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "qed.h"),
                                                                 os.path.abspath(__file__)]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force=False, verbose=False, checks=False):
    """Compile every CUDA/C++ source of the library and link libqed.so (with checks=True the
    debug build with device bounds checks, libqed_checks.so); returns its path."""
    lib = LIB_CHECKS if checks else LIB
    if not force and not _stale(lib):
        return lib
    os.makedirs(BUILD_CHECKS if checks else BUILD, exist_ok=True)
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose, checks), srcs))
    objs = [o for o, _ in results]
    if verbose:
        for (_, log), s in zip(results, srcs):
            if log.strip():
                print(f"--- {s}\n{log}")
    tmp = lib + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp] + ARCH + objs + ["-lcudart", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checks="--checks" in sys.argv))
