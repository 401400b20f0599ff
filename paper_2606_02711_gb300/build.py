"""Builds liblym1.so (the CUDA library behind include/lym1.h) in-tree for sm_103a.

Translation units compiled in parallel, then linked:
  csrc/lym1_tables.cpp        host per-bin tables (g++, no FMA contraction)
  csrc/lym1_api.cu            C ABI host code
  csrc/lym1_kernels_det.cu    FP64 fixed-order kernels (-fmad=false)
  csrc/lym1_kernels_fast.cu   dispatch to the FP64 / mixed policies
  csrc/lym1_pol_*.cu          every kernel of one of those policies (one unit each)
  csrc/lym1_noalloc.cu        allocation-free energy reduction
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "liblym1.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")

SOURCES = ["lym1_tables.cpp", "lym1_api.cu", "lym1_kernels_det.cu", "lym1_kernels_fast.cu",
           "lym1_pol_f64.cu", "lym1_pol_mix.cu", "lym1_pol_mixf.cu", "lym1_noalloc.cu"]
HEADERS = ["lym1_internal.h", "lym1_kernels.cuh", "lym1_policies.h", "lym1_pol_unit.cuh"]
# FMA contraction, FP32 flush-to-zero and approximate FP32 divide/sqrt
FAST_UNITS = ("lym1_kernels_fast.cu", "lym1_pol_f64.cu", "lym1_pol_mix.cu", "lym1_pol_mixf.cu")


def _cmd(src: str) -> list[str]:
    path = os.path.join(CSRC, src)
    obj = os.path.join(BUILD, src + ".o")
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if src.endswith(".cpp"):
        return ["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-ffp-contract=off", "-fno-fast-math",
                *inc, "-c", path, "-o", obj]
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-ffp-contract=off", *inc, "-c", path, "-o", obj]
    if src == "lym1_kernels_det.cu":
        cmd.insert(1, "-fmad=false")
    if src in FAST_UNITS:
        # FP32 policies: flush subnormals, approximate FP32 divide/sqrt (FP64
        # arithmetic is not affected by these flags)
        cmd[1:1] = ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"]
    return cmd


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + HEADERS
    paths = [os.path.join(CSRC, s) for s in deps] + [os.path.join(ROOT, "include", "lym1.h")]
    return any(os.path.getmtime(p) > t for p in paths)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, [_cmd(s) for s in SOURCES]))
    objs = [os.path.join(BUILD, s + ".o") for s in SOURCES]
    run([NVCC, *ARCH, "-shared", "-o", LIB + ".tmp", *objs, "-lpthread"])
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
