"""Build libcfsim.so in-tree for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_1707_02423_gb300/libcfsim.so`` against the shared CUDA runtime (the one
torch loads).  Rebuilds only what changed.  ``python -m paper_1707_02423_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcfsim.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["api.cu", "plan.cu", "forward.cu", "backward.cu", "misc.cu", "static_ws.cu", "probe.cu", "graph.cu", "autotune.cu", "match_opt.cu", "distances.cu", "ward.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-I", INCLUDE,
         "-I", CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _headers_mtime() -> float:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(INCLUDE, "cfsim.h"))
    return max(os.path.getmtime(h) for h in hs)


def _compile(src: str, extra: list[str], verbose: bool) -> str:
    obj = os.path.join(BUILD, src + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        print(r.stdout, r.stderr, flush=True)
    return obj


# Build variants: the product library, and a debug build whose kernels check
# layouts, slots and staged indices (-DCF_DEBUG_BOUNDS; a failed check sets
# the status word), loaded by setting CFSIM_LIBRARY to its path.
VARIANTS = {None: (BUILD, LIB, []),
            "debug_bounds": (os.path.join(HERE, "_build_debug"), os.path.join(HERE, "libcfsim_debug.so"),
                             ["-DCF_DEBUG_BOUNDS"])}


def build(verbose: bool = False, force: bool = False, extra: list[str] | None = None,
          variant: str | None = None) -> str:
    """Compile every CUDA source for sm_103a and link the library (libcfsim.so,
    or the variant's); returns its path."""
    global BUILD, LIB
    bdir, lib, vflags = VARIANTS[variant]
    if variant is not None:
        saved = (BUILD, LIB)
        BUILD, LIB = bdir, lib
        try:
            return build(verbose, force, list(extra or []) + vflags, None)
        finally:
            BUILD, LIB = saved
    extra = list(extra or [])
    os.makedirs(BUILD, exist_ok=True)
    hdr_t = _headers_mtime()
    todo = []
    for s in SOURCES:
        obj = os.path.join(BUILD, s + ".o")
        src_t = os.path.getmtime(os.path.join(CSRC, s))
        if force or (extra and BUILD == VARIANTS[None][0]) or not os.path.exists(obj) or \
                os.path.getmtime(obj) < max(src_t, hdr_t):
            todo.append(s)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(lambda s: _compile(s, extra, verbose), todo))
    objs = [os.path.join(BUILD, s + ".o") for s in SOURCES]
    if todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + ".tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None
    variant = "debug_bounds" if "--debug-bounds" in sys.argv else None
    print(build(verbose=v, force="--force" in sys.argv, extra=extra, variant=variant))
