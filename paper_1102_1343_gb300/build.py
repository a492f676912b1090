"""Build the CUDA library libwrffire_gb300.so in-tree for sm_103a.

Compiles the translation units of csrc/ in parallel with nvcc (one
-gencode, arch=compute_103a,code=sm_103a) and links a shared library with the
CUDA runtime linked statically.  ptxas resource usage is written to
_build/ptxas.log.  build(checked=True) builds the same sources with
-DFIRE_BOUNDS_CHECK (every global index of the step kernels checked, a bad
one reported as FIRE_ERR_BOUNDS) into libwrffire_gb300_checked.so, for tests.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libwrffire_gb300.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libwrffire_gb300_checked.so")
SOURCES = ["step_f32.cu", "step_f64.cu", "coeffs.cu", "context.cu", "noalloc.cu",
           "ensemble.cu", "adjoint.cu", "coupling.cu", "step_warp4.cu"]
HEADERS = ["step_kernel.cuh", "march_kernel.cuh", "warp_kernel.cuh", "warp4_kernel.cuh", "pair_math.cuh", "fire_device.cuh", "fire_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
              "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _deps():
    inc = os.path.join(os.path.dirname(HERE), "include", "wrffire.h")
    return [os.path.join(CSRC, h) for h in HEADERS] + [inc, os.path.abspath(__file__)]


def _stale(target, inputs):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(p) > t for p in inputs)


def _compile(src, build_dir=BUILD, defines=()):
    obj = os.path.join(build_dir, src.replace(".cu", ".o"))
    inputs = [os.path.join(CSRC, src)] + _deps()
    if not _stale(obj, inputs):
        return obj, ""
    cmd = ([nvcc()] + ARCH + NVCC_FLAGS + list(defines) +
           ["-c", os.path.join(CSRC, src), "-o", obj + ".tmp"])
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{p.stdout}\n{p.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj, p.stdout + p.stderr


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    build_dir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    defines = ["-DFIRE_BOUNDS_CHECK"] if checked else []
    os.makedirs(build_dir, exist_ok=True)
    if force:
        for f in os.listdir(build_dir):
            if f.endswith(".o"):
                os.remove(os.path.join(build_dir, f))
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, build_dir, defines), SOURCES))
    objs = [o for o, _ in results]
    logs = "".join(l for _, l in results)
    if logs:
        with open(os.path.join(build_dir, "ptxas.log"), "w") as f:
            f.write(logs)
        if verbose:
            print(logs)
    if _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"link failed:\n{p.stdout}\n{p.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
