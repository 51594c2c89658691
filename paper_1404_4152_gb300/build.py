"""Compile the CUDA library (libswgb300.so) in-tree for sm_103a.

Each translation unit compiles in its own nvcc process, in parallel, and the
objects are linked into ``paper_1404_4152_gb300/_build/libswgb300.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB_NAME = "libswgb300.so"
DEBUG_LIB_NAME = "libswgb300_debug.so"  # built with -DSW_DEBUG_BOUNDS (checked accesses)

SOURCES = ["sw_wavefront.cu", "sw_rescore.cu", "sw_topk.cu", "sw_api.cu", "sw_search.cu",
           "sw_noalloc.cu", "sw_server.cu", "sw_tune.cu", "sw_align.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def lib_path(debug: bool = False) -> str:
    return os.path.join(BUILD, DEBUG_LIB_NAME if debug else LIB_NAME)


def _digest(paths) -> str:
    h = hashlib.sha256()
    for p in sorted(paths):
        h.update(p.encode())
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".h", ".cuh", ".cpp"))]
    files.append(os.path.join(INCLUDE, "sw.h"))
    return files


def build(verbose: bool = False, force: bool = False, debug: bool = False) -> str:
    """Build the library if any source changed; returns the .so path. ``debug`` builds
    the bounds-checked variant (every checked device access records its site in an
    error word and is skipped when out of bounds; see sw_db_debug_check)."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp_debug.txt" if debug else "stamp.txt")
    extra = ["-DSW_DEBUG_BOUNDS"] if debug else []
    digest = _digest(_inputs()) + ("-debug" if debug else "")
    out = lib_path(debug)
    if not force and os.path.exists(out) and os.path.exists(stamp):
        if open(stamp).read().strip() == digest:
            return out
    cmds = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", "_dbg.o" if debug else ".o"))
        objs.append(obj)
        cmds.append([nvcc(), *ARCH, *FLAGS, *extra, "-I", INCLUDE, "-I", CSRC, "-c",
                     os.path.join(CSRC, src), "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        for cmd, r in ex.map(run, cmds):
            if verbose and r.stderr:
                sys.stderr.write(r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    tmp = out + f".tmp{os.getpid()}"
    link = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-lpthread",
            "-ldl"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(link)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    with open(stamp, "w") as f:
        f.write(digest)
    return out


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
