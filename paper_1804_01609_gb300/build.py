"""Build the CUDA library librbfsl.so in-tree for sm_103a (GB300).

Every .cu under csrc/ is compiled in parallel (with relocatable device code, except the units in
WHOLE_PROGRAM) and linked by
nvcc into paper_1804_01609_gb300/_build/librbfsl.so. Rebuilds only when a source or header
is newer than the library.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "librbfsl.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Translation units compiled as whole programs (no relocatable device code). global_tc.cu
# references no device symbol of another unit; built with -rdc=true, its tcgen05 kernel returned
# wrong accumulators on sm_103a (a standalone build of the same source reproduces this), built
# whole-program it matches the FP64 evaluation to the split-TF32 bound.
WHOLE_PROGRAM = {"global_tc.cu"}


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    # -fmad=false: no implicit contraction of a*b+c into FMA. The hot loops use explicit fma();
    # everything else is rounded operation by operation, so the same device code gives the same
    # bits in every kernel it is inlined into (single problem, batch, server).
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-rdc=true", "-fmad=false", "-Xcompiler", "-fPIC",
                     "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC] + list(extra_flags)

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
        flags = common
        if os.path.basename(src) in WHOLE_PROGRAM:
            # without -rdc the constant-memory tables declared extern in common.cuh become a
            # (unused) static definition of this unit; nvcc says so in warning 20044
            flags = [f for f in common if f != "-rdc=true"] + ["-diag-suppress", "20044"]
        cmd = [cc] + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return obj

    srcs = _sources()
    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cc] + ARCH + ["-shared", "-rdc=true", "-Xcompiler", "-fPIC", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
