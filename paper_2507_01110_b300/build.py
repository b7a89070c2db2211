"""Compile liblodgs.so (the CUDA path) for sm_103a with nvcc, in the package folder.

Translation units that take float32 decisions (scene build, LoD selection,
projection) are compiled with -fmad=false so that every expression is rounded
as written; host code is compiled with -ffp-contract=off for the same reason.

Build knobs (environment): LODGS_DEFINES adds preprocessor definitions (for
example "LODGS_BWD_F32X2=0 LODGS_FWD_F32X2=0" for the blends' scalar loops);
objects then go to their own folder.  LODGS_LIBRARY, if set, is where the
library is written (and where the binding loads it from).
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
DEFINES = os.environ.get("LODGS_DEFINES", "").split()
BUILD = os.path.join(ROOT, "_build", "_".join(d.replace("=", "-") for d in DEFINES)) if DEFINES else \
    os.path.join(ROOT, "_build")
LIB = os.environ.get("LODGS_LIBRARY", os.path.join(PKG, "liblodgs.so"))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                 "-I", os.path.join(ROOT, "include"), "--expt-relaxed-constexpr"]
EXACT = {"scene.cu", "select.cu", "project.cu", "abi.cu"}     # no FMA contraction
SOURCES = ["abi.cu", "scene.cu", "select.cu", "project.cu", "raster.cu", "sort.cu", "noalloc.cu", "cache.cu", "batch.cu",
           "loss.cu", "adam.cu", "densify.cu"]


def _newer(src_paths, out):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(p) > t for p in src_paths)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(os.path.dirname(LIB) or ".", exist_ok=True)
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    hdrs.append(os.path.join(ROOT, "include", "lodgs.h"))
    jobs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        objs.append(obj)
        if force or _newer([src] + hdrs + [__file__], obj):
            flags = COMMON + (["-fmad=false"] if s in EXACT else []) + [f"-D{d}" for d in DEFINES]
            jobs.append([NVCC] + flags + ["-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)

    with ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        list(ex.map(run, jobs))
    if force or jobs or _newer(objs, LIB):
        run([NVCC] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
