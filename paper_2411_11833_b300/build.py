"""Compile libtamp.so in-tree for sm_103a (B300) with nvcc."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SOURCES = [os.path.join(HERE, "csrc", f) for f in ("tamp_kernels.cu", "tamp_api.cu", "tamp_mlp.cu")]
HEADERS = [os.path.join(HERE, "csrc", "tamp_dev.cuh"), os.path.join(ROOT, "include", "tamp.h")]
OUT = os.path.join(HERE, "lib", "libtamp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# FP32 division and square root in the approximate forms (within 2 ulp, not
# correctly rounded): the IEEE forms cost the fused optimisation kernel 11% of
# its throughput, and 2 ulp is far inside the parity tolerances (1e-4 relative
# on costs, 1e-3 on gradients).  FP32 subnormals (below 1.2e-38, far under any
# length, angle or gradient the method forms) flush to zero: another 1%.
# Transcendentals (sincosf, atan2f) stay precise.
MATH = ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]


def nvcc_command(out: str = OUT, extra=()):
    return (["nvcc", "-O3", "-std=c++17", *ARCH, *MATH, "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
             "-I", os.path.join(ROOT, "include"), *extra, "-o", out, *SOURCES])


def up_to_date(out: str = OUT) -> bool:
    if not os.path.exists(out):
        return False
    t = os.path.getmtime(out)
    return all(os.path.getmtime(s) <= t for s in SOURCES + HEADERS + [os.path.abspath(__file__)])


def build_library(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    if not force and up_to_date():
        return OUT
    cmd = nvcc_command(extra=["-Xptxas", "-v"] if verbose else [])
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stdout + res.stderr)
    if verbose:
        print(res.stdout + res.stderr)
    return OUT


if __name__ == "__main__":
    import sys
    print(build_library(force="--force" in sys.argv, verbose="-v" in sys.argv))
