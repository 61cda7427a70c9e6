"""Build the gbqr shared library (libgbqr.so) for sm_103a, in-tree.

Each .cu translation unit is compiled in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a), then linked into
paper_2212_01997_gb300/libgbqr.so.  Object files go to _build/.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libgbqr.so")
# (source, object, defines): mixed.cu is compiled three times, once per
# configuration of the one-tile split-precision kernel; big.cu holds the tiled
# kernel for subgraphs above 128 orbitals
SOURCES = [("api.cu", "api", []), ("graph.cu", "graph", []), ("partition.cu", "partition", []),
           ("density.cu", "density", []), ("mixed.cu", "mixed", []),
           ("mixed.cu", "mixed_listed", ["-DGB_SPLIT_LIST=1"]),
           ("mixed.cu", "mixed_small", ["-DGB_SPLIT_NPMAX=64", "-DGB_SPLIT_LIST=1"]),
           ("big.cu", "big", []), ("charges.cu", "charges", []), ("eigen.cu", "eigen", []),
           ("krylov.cu", "krylov", [])]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the gbqr CUDA library cannot be built")


def _compile(unit: tuple, extra: list[str]) -> str:
    src, name, defines = unit
    obj = os.path.join(BUILD, name + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-I", INCLUDE, "-I", CSRC, *defines, "-c", os.path.join(CSRC, src), "-o", obj, *extra]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    return obj


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "gbqr.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile and link libgbqr.so if a source is newer than the library."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra or [])
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None)
