"""Build libmpgabor.so in-tree for sm_103a (GB300) with plain nvcc.

Each .cu file of csrc/ is compiled in parallel, then linked into
paper_2202_12380_gb300/_build/libmpgabor.so.  nvcc cross-compiles without a
GPU, so this runs on any host with CUDA 13.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmpgabor.so")
# the same library with every MP-loop access bounds-checked (-DMP_CHECK_BOUNDS),
# for the GPU tests
CHECKED_DIR = os.path.join(OUT_DIR, "checked")
LIB_CHECKED = os.path.join(CHECKED_DIR, "libmpgabor.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(lib, deps):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=None, checked: bool = False) -> str:
    out_dir = CHECKED_DIR if checked else OUT_DIR
    lib = LIB_CHECKED if checked else LIB
    os.makedirs(out_dir, exist_ok=True)
    srcs = sources()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "mpgabor.h"))
    if not force and not _stale(lib, srcs + headers + [os.path.abspath(__file__)]):
        return lib
    nv = nvcc()
    flags = FLAGS + list(extra or []) + (["-DMP_CHECK_BOUNDS"] if checked else [])

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [nv] + ARCH + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nv] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> list:
    """Both libraries (the product and its bounds-checked twin), built side
    by side."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        return list(ex.map(lambda c: build(force=force, checked=c), (False, True)))


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
