"""Build the sm_103a shared library ``libsbm.so`` in-tree.

Every translation unit is compiled in parallel (nvcc for .cu, g++ for plain
C++), then linked into ``paper_2507_17053_gb300/libsbm.so``.  Objects go to
``_build/`` at the repository root.  Host C++ is compiled with
``-ffp-contract=off`` so the active-cell decisions do not depend on whether
the host compiler fuses multiply-adds (x86 vs Arm).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libsbm.so")

ARCH = "-gencode=arch=compute_103a,code=sm_103a"
# the device set-up shares its level-set arithmetic with the host set-up and
# must round like it: no fused multiply-adds there
PER_FILE = {"setup_gpu.cu": ["--fmad=false"]}


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cu", ".cpp")))


def _compile(src: str, extra: list[str]) -> str:
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    inc = [f"-I{INCLUDE}", f"-I{CSRC}"]
    if src.endswith(".cu"):
        cmd = [_nvcc(), ARCH, "-lineinfo", "-O3", "-std=c++17", "-c", src, "-o", obj,
               "-Xcompiler", "-fPIC,-ffp-contract=off", "--expt-relaxed-constexpr", *inc, *extra,
               *PER_FILE.get(os.path.basename(src), [])]
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall", "-c", src,
               "-o", obj, f"-I{os.path.join(os.path.dirname(_nvcc()), '..', 'include')}", *inc]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(verbose: bool = False, extra_nvcc: list[str] | None = None) -> str:
    """Compile and link; returns the path of libsbm.so."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(16, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra_nvcc or []), srcs))
    tmp = LIB + ".tmp"
    cmd = [_nvcc(), ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    build(verbose=True)
