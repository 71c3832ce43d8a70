"""Build the CUDA library ``_build/libfvgb.so`` in-tree for sm_103a with nvcc.

Translation units are compiled in parallel; the FP64 step kernels are
compiled twice from one source, without (``fv_fp64_exact``) and with
(``fv_fp64_fma``) fused multiply-add contraction.  Rebuilds only when a
source is newer than the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfvgb.so")
PROBE = os.path.join(BUILD, "fp64_probe")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
          "-Xcompiler", "-fvisibility=hidden",
          "-I", CSRC, "-I", INCLUDE]

# (object name, source, extra flags)
UNITS = [
    ("fv_step_fp64_exact.o", "fv_step_kernels.cu", ["--fmad=false", "-DFV_NS=fv_fp64_exact"]),
    ("fv_step_fp64_fma.o", "fv_step_kernels.cu", ["--fmad=true", "-DFV_NS=fv_fp64_fma",
                                                         "-DFV_NEWTON_DIVSQRT"]),
    ("fv_fused64_exact.o", "fv_fused64_kernels.cu", ["--fmad=false", "-DFV_NS=fv_fp64_exact"]),
    ("fv_fused64_fma.o", "fv_fused64_kernels.cu", ["--fmad=true", "-DFV_NS=fv_fp64_fma",
                                                   "-DFV_NEWTON_DIVSQRT"]),
    ("fv_fused_ff.o", "fv_fused_ff_kernels.cu", ["--fmad=false", "-DFV_NEWTON_DIVSQRT"]),
    ("fv_step_fp32.o", "fv_step32_kernels.cu", ["--fmad=false"]),
    ("fv_aux.o", "fv_aux.cu", ["--fmad=false"]),
    ("fv_core.o", "fv_core.cu", ["--fmad=false"]),
    ("fv_noalloc.o", "fv_noalloc.cu", ["--fmad=false"]),
    ("fv_batch.o", "fv_batch.cu", ["--fmad=false"]),
    ("fv_learned.o", "fv_learned.cu", ["--fmad=true"]),
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfvgb.so")


def _sources():
    out = []
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cuh", ".h")) and f != "fp64_probe.cu":
                out.append(os.path.join(d, f))
    out.append(os.path.abspath(__file__))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(PROBE):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(PROBE))
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_unit(unit):
        obj, src, extra = unit
        cmd = [cc, *ARCH, *COMMON, *extra, "-c", os.path.join(CSRC, src),
               "-o", os.path.join(BUILD, obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    def compile_probe():
        cmd = [cc, *ARCH, "-O3", "-std=c++17", os.path.join(CSRC, "fp64_probe.cu"), "-o", PROBE]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on fp64_probe.cu:\n{r.stderr}")

    with ThreadPoolExecutor(max_workers=len(UNITS) + 1) as ex:
        probe = ex.submit(compile_probe)
        objs = list(ex.map(compile_unit, UNITS))
        probe.result()
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[os.path.join(BUILD, o) for o in objs]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
