"""Build libgks.so in-tree for sm_103a (nvcc, one -gencode, parallel TUs).

    python -m paper_2508_19911_gb300.build [--force]

Output: paper_2508_19911_gb300/_build/libgks.so (git-ignored). Rebuilds only
when a source is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libgks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["flux.cu", "recon.cu", "recon_fp64.cu", "update.cu", "capi.cu", "noalloc.cu", "mlp.cu", "ensemble.cu", "peak.cu",
              "ensemble_step.cu", "recon_lines.cu"]
CPP_SOURCES = ["tables.cpp"]
HEADERS = ["basis.h", "common.cuh", "ff.cuh", "recon_common.cuh", "flux_device.cuh",
           "recon_fp64_device.cuh", "recon_mixed_device.cuh", "update_device.cuh"]
# recon.cu (the mixed-precision reconstruction): no implicit multiply-add
# contraction (only explicit fmaf), so that every kernel inlining the same
# reconstruction rounds identically (the learned indicator's never-skip
# limit equals the plain kernel bit for bit; ptxas would otherwise fuse
# differently in each kernel's context). recon_fp64.cu keeps contraction.
EXTRA_FLAGS = {"recon.cu": ["-fmad=false"]}
COMPILE_TIMEOUT = 900


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _deps():
    files = [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES + HEADERS]
    files.append(os.path.join(ROOT, "include", "gks.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def _compile(src: str, obj: str) -> None:
    cmd = [nvcc()] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                             "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
    if src.endswith(".cpp"):
        cmd += ["-x", "c++"]
    cmd += EXTRA_FLAGS.get(os.path.basename(src), [])
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=COMPILE_TIMEOUT)
    if r.returncode != 0:
        raise RuntimeError(f"compiling {os.path.basename(src)} failed:\n{r.stderr[-4000:]}")


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    for f in CU_SOURCES + CPP_SOURCES:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, os.path.splitext(f)[0] + ".o")
        jobs.append((src, obj))
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1)) as ex:
        futs = [ex.submit(_compile, s, o) for s, o in jobs]
        for fu in futs:
            fu.result()
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for _, o in jobs]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=COMPILE_TIMEOUT)
    if r.returncode != 0:
        raise RuntimeError("linking libgks.so failed:\n" + r.stderr[-4000:])
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
