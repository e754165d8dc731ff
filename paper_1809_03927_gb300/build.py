"""Build ``libdose.so`` (the C-ABI CUDA engine) in-tree for sm_103a.

Each translation unit under ``csrc/`` is compiled by nvcc in parallel and
linked into ``paper_1809_03927_gb300/lib/libdose.so`` with the CUDA runtime
linked statically.  No cmake; a rebuild compiles only changed sources.
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
OUT_DIR = os.path.join(PKG, "lib")
OBJ_DIR = os.path.join(PKG, "lib", "obj")
LIB = os.path.join(OUT_DIR, "libdose.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "transport.cu", "timeline.cu", "emtm.cu", "dim.cu", "dvf.cu", "lut.cpp", "noalloc.cu", "serve.cpp", "peaks.cu"]
# Per-source flags.  The transport flushes single-precision subnormals: none
# of its values comes near 1e-38 (energies, ranges, positions, directions,
# weights and the uniforms are all of order 1e-7 or more), so results do not
# change, and the approximate reciprocal, square root, logarithm and sine
# need no scaling of subnormal inputs around each hardware instruction.
SOURCE_FLAGS = {"transport.cu": ["-ftz=true"]}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdose")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                   "-I", CSRC, "-I", INCLUDE, *extra]


def _deps_mtime(src: str) -> float:
    heads = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    heads.append(os.path.join(INCLUDE, "dose.h"))
    heads.append(os.path.abspath(__file__))            # flags live here
    return max([os.path.getmtime(src)] + [os.path.getmtime(h) for h in heads])


def _compile(src: str, verbose: bool, extra) -> str:
    obj = os.path.join(OBJ_DIR, os.path.splitext(os.path.basename(src))[0] + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= _deps_mtime(src):
        return obj
    cmd = [nvcc(), "-c", src, "-o", obj + ".tmp"] + _flags(list(extra) + SOURCE_FLAGS.get(os.path.basename(src), []))
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        sys.stderr.write(r.stdout + r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, extra=()) -> str:
    """Compile every source (in parallel) and link ``libdose.so``."""
    os.makedirs(OBJ_DIR, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, extra), srcs))
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(o) for o in objs):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-shared", "-o", tmp, *objs] + ARCH + ["-cudart", "static", "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
