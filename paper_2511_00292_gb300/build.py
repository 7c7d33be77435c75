"""Build the CUDA library libeig3.so in-tree for GB300 (sm_103a).

The translation units are compiled in parallel with nvcc and linked into
``paper_2511_00292_gb300/_build/libeig3.so`` (static CUDA runtime, no torch
dependency: the C ABI takes plain pointers).  ptxas resource usage of every
kernel is kept next to the objects (``_build/ptxas_<unit>.txt``).  The
throughput loops that give the benchmark its FP64 / FP32 peaks
(``csrc/eig3_peaks.cu``) go into a library of their own,
``_build/libeig3_peaks.so``, which the eig3 ABI does not include.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libeig3.so")
PEAKS_LIB = os.path.join(BUILD, "libeig3_peaks.so")
PEAKS_UNIT = "eig3_peaks.cu"

UNITS = ["eig3_api.cu", "eig3_f64.cu", "eig3_f32c.cu", "eig3_mohr_coulomb.cu", "eig3_variants.cu",
         "eig3_guard.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
          "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libeig3.so")


def _deps_mtime() -> float:
    files = glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def _compile(unit: str) -> str:
    src = os.path.join(CSRC, unit)
    obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
    cmd = [nvcc(), *ARCH, *CFLAGS, "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    with open(os.path.join(BUILD, f"ptxas_{unit.replace('.cu', '')}.txt"), "w") as f:
        f.write(res.stderr)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {unit}:\n{res.stderr[-4000:]}")
    return obj


def build(force: bool = False) -> str:
    """Compile (if stale) and link libeig3.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    fresh = all(os.path.exists(p) and os.path.getmtime(p) >= _deps_mtime()
                for p in (LIB, PEAKS_LIB))
    if not force and fresh:
        return LIB
    with ThreadPoolExecutor(max_workers=len(UNITS) + 1) as ex:
        objs = list(ex.map(_compile, UNITS + [PEAKS_UNIT]))
    for lib, parts in ((LIB, objs[:-1]), (PEAKS_LIB, objs[-1:])):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *parts]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stderr[-4000:]}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
