"""Build libibfsa.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel; the strict-arithmetic units (the FP64 stage and the
plate) get --fmad=false so that no multiply and add are fused there, and the plate's host code
(the clamp motion) -ffp-contract=off for the same reason.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libibfsa.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
          "--expt-relaxed-constexpr"]

UNITS = {
    "api.cu": ["-Xcompiler", "-ffp-contract=off"],
    "stage_fp64_strict.cu": ["--fmad=false"],
    "stage_fp64_fast.cu": ["--fmad=true"],
    "stage_fp32.cu": ["--fmad=true"],
    "mlp.cu": ["--fmad=true"],
    "noalloc.cu": [],
    "stats.cu": [],
    "plate.cu": ["--fmad=false", "-Xcompiler", "-ffp-contract=off"],
}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources_mtime() -> float:
    m = 0.0
    for d in (CSRC, os.path.join(os.path.dirname(HERE), "include")):
        for f in os.listdir(d):
            m = max(m, os.path.getmtime(os.path.join(d, f)))
    return m


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(item):
        src, flags = item
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *flags, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS.items()))
    tmp = LIB + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


PIPE_RATES = os.path.join(HERE, "pipe_rates")


def build_pipe_rates(force: bool = False) -> str:
    """The standalone pipe-throughput probe (csrc/pipe_rates.cu): the FP64 and FP32 fused
    multiply-add and the multi-function unit's rates the kernels' rooflines are quoted against."""
    src = os.path.join(CSRC, "pipe_rates.cu")
    if not force and os.path.exists(PIPE_RATES) and os.path.getmtime(PIPE_RATES) >= os.path.getmtime(src):
        return PIPE_RATES
    cmd = [nvcc(), *ARCH, "-O3", "-std=c++17", src, "-o", PIPE_RATES]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on pipe_rates.cu:\n{r.stdout}\n{r.stderr}")
    return PIPE_RATES


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, extra=tuple(sys.argv[1:])))
