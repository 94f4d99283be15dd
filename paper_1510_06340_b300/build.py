"""Build libhydro.so (the C-ABI solver library) for B300 (sm_103a) with nvcc.

The library is built in-tree next to this file so that it travels with the
repository; objects go to _build/.  `python -m paper_1510_06340_b300.build`
rebuilds when a source is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
OUT = os.environ.get("HYDRO_LIB_OUT", os.path.join(HERE, "libhydro.so"))
BUILD = os.environ.get("HYDRO_BUILD_DIR", os.path.join(HERE, "_build"))
# extra nvcc flags (e.g. -DHY_SWEEP_MAXNREG=112) for launch-shape experiments
EXTRA = os.environ.get("HYDRO_NVCC_FLAGS", "").split()
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
BASE = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + SRC, "-I" + INC]
# float sweeps use approximate sqrt/divide and flush denormals (a few ulp, far
# inside the FP32 tolerance)
FAST = {"sweep_f32.cu", "sweep_mixed.cu", "unsplit_f32.cu", "unsplit_mixed.cu"}
FAST_FLAGS = ["-ftz=true", "-prec-div=false", "-prec-sqrt=false", "-DHY_FTZ"]
NOFMAD = set()   # units compiled with -fmad=false (none)


def _sources():
    return sorted(glob.glob(os.path.join(SRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(SRC, "*.cuh")) + glob.glob(
        os.path.join(SRC, "*.h")) + [os.path.join(INC, "hydro.h"), __file__]


def needs_build() -> bool:
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    return any(os.path.getmtime(p) > t for p in _deps())


def _compile(src: str) -> str:
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    flags = list(BASE) + EXTRA
    if os.path.basename(src) in FAST:
        flags += FAST_FLAGS
    if os.path.basename(src) in NOFMAD:
        flags.append("-fmad=false")
    cmd = [NVCC] + flags + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = True) -> str:
    if not force and not needs_build():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(_compile, srcs))
    tmp = OUT + f".tmp{os.getpid()}"
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    if verbose:
        print(f"built {OUT}", file=sys.stderr)
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv)
