"""Build libhpmc.so (CUDA, sm_103a) in-tree with nvcc.

Translation units are compiled in parallel into ``_build/`` and linked into
``_build/libhpmc.so``.  ``-fmad=false`` keeps every FP64 operation of the
decision contract a single IEEE rounding (FP32 filter code uses explicit
fused multiply-adds); ``-ffp-contract=off`` does the same for host code.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhpmc.so")
# trace variant (-DHPMC_TRACE): per-warp clock64() phase stamps in the set kernels
BUILD_TRACE = os.path.join(HERE, "_build_trace")
LIB_TRACE = os.path.join(BUILD_TRACE, "libhpmc.so")
UNITS = ["hpmc.cu", "set2d_f32.cu", "set2d_direct.cu", "set2d_f64.cu", "set3d.cu", "set3d_f32.cu", "set3d_f64.cu",
         "set3d_f32_nv20.cu", "set3d_f64_nv20.cu", "selects.cu", "noalloc.cu", "pairtest.cu", "peaks.cu", "pressure.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC,-ffp-contract=off",
         "-I", INCLUDE]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhpmc.so")


def _sources():
    return [os.path.join(CSRC, u) for u in UNITS if os.path.exists(os.path.join(CSRC, u))]


def _newest_input() -> float:
    t = 0.0
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            t = max(t, os.path.getmtime(os.path.join(d, f)))
    return max(t, os.path.getmtime(__file__))


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          trace: bool = False) -> str:
    bdir, lib = (BUILD_TRACE, LIB_TRACE) if trace else (BUILD, LIB)
    if trace:
        extra = list(extra or []) + ["-DHPMC_TRACE"]
    os.makedirs(bdir, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest_input():
        return lib
    cc = nvcc()
    srcs = _sources()
    objs = [os.path.join(bdir, os.path.basename(s).replace(".cu", ".o")) for s in srcs]

    def one(pair):
        s, o = pair
        cmd = [cc, *ARCH, *FLAGS, *(extra or []), "-c", s, "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {s}:\n{r.stdout}\n{r.stderr}")
        return r.stdout + r.stderr

    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        logs = list(ex.map(one, zip(srcs, objs)))
    if verbose:
        for lg in logs:
            print(lg)
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None,
                trace="--trace" in sys.argv))
