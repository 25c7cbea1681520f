"""Compile liborrb.so in-tree for sm_103a (nvcc, no fast-math).

    python -m paper_1906_11633_b300.build [--force]
"""

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
SOURCES = ["orrb_api.cpp", "orrb_render.cu", "orrb_shadow_table.cu", "orrb_post.cu", "orrb_backward.cu"]
HEADERS = [os.path.join(CSRC, "orrb_internal.h"), os.path.join(CSRC, "orrb_shading.cuh"), os.path.join(ROOT, "include", "orrb.h")]
LIB = os.path.join(HERE, "liborrb.so")
PEAK_SRC = os.path.join(CSRC, "orrb_fp32_peak.cu")
PEAK_LIB = os.path.join(HERE, "libfp32peak.so")
NVCC_FLAGS = ["-std=c++17", "-O3", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-Xcompiler", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in [os.path.join(CSRC, s) for s in SOURCES] + HEADERS)


def build_peak(force: bool = False, verbose: bool = False) -> str:
    """The FP32 peak probe (measurement infrastructure, its own library)."""
    if force or not os.path.exists(PEAK_LIB) or os.path.getmtime(PEAK_SRC) > os.path.getmtime(PEAK_LIB):
        tmp = PEAK_LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc(), *NVCC_FLAGS, "-o", tmp, PEAK_SRC]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        os.replace(tmp, PEAK_LIB)
    return PEAK_LIB


def build(force: bool = False, verbose: bool = False) -> str:
    build_peak(force, verbose)
    if force or stale():
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc(), *NVCC_FLAGS, "-o", tmp] + [os.path.join(CSRC, s) for s in SOURCES]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
