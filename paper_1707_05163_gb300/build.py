"""Compile the CUDA library in-tree for sm_103a (no cmake, no torch extension).

Each translation unit compiles in parallel with nvcc; the FP64 advection unit
gets -fmad=false so its multiplies and adds round separately, in source order.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
# PG_BUILD_DIR / PG_MAXRREG: build elsewhere / cap registers of the FP32
# advection unit (tuning experiments); defaults build the library in-tree.
OUT_DIR = os.environ.get("PG_BUILD_DIR", os.path.join(HERE, "_build"))
LIB = os.path.join(OUT_DIR, "libparcels_gb.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
BASE = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
        "--expt-relaxed-constexpr", "-I", CSRC, "-I", INCLUDE]
UNITS = {
    "capi.cu": [],
    "field_store.cu": [],
    "sort.cu": [],
    "advect_f64.cu": ["-fmad=false"],
    "advect_cell.cu": [],
    "moments_noalloc.cu": [],
    "batch.cu": [],
    "mlp.cu": [],
    "mlp_tc.cu": [],
    "mlp_fused.cu": [],
    "surrogate.cu": [],
    "advect_f32.cu": ([f"-maxrregcount={os.environ['PG_MAXRREG']}"]
                      if os.environ.get("PG_MAXRREG") else []),
    "advect_f32_ext.cu": [],
    "probe.cu": [],
    "output.cu": [],
}


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build the library")
    return p


def _deps_mtime() -> float:
    m = 0.0
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            m = max(m, os.path.getmtime(os.path.join(d, f)))
    return m


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    cc = nvcc()

    def compile_unit(item):
        src, extra = item
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        cmd = [cc, *BASE, *ARCH, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(compile_unit, UNITS.items()))
    if verbose:
        for _, err in results:
            print(err)
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cc, "-shared", *ARCH, "-o", tmp, *[o for o, _ in results], "-lcuda"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
