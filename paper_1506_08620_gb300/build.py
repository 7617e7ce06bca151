"""Compile the CUDA library libds.so in-tree for sm_103a.

Each translation unit under csrc/ is compiled in parallel with nvcc
(``-gencode arch=compute_103a,code=sm_103a``), then linked into
``paper_1506_08620_gb300/libds.so`` with the CUDA runtime linked statically.
Objects go to ``paper_1506_08620_gb300/_build/`` (git-ignored).

``build(bounds=True)`` compiles the range-checking variant
``libds_bounds.so`` (``-DDS_DEBUG_BOUNDS``, objects in ``_build_bounds/``):
every table and knot gather of the search kernels checks its index, and an
index out of range is recorded in the handle's device error word instead of
being read.  The package loads it when ``DS_LIBRARY=bounds``.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libds.so")
BOUNDS_OUT_DIR = os.path.join(PKG, "_build_bounds")
BOUNDS_LIB = os.path.join(PKG, "libds_bounds.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + [
    "-O3", "-std=c++17", "-lineinfo", "--fmad=false", "-ftz=false", "-prec-div=true", "-prec-sqrt=true",
    "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", "-Xcompiler", "-fvisibility=hidden",
    "-Xptxas", "-warn-spills", "-I" + INCLUDE, "-I" + CSRC,
]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hs + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]


def _compile(src, verbose_ptxas=False, bounds=False):
    obj = os.path.join(BOUNDS_OUT_DIR if bounds else OUT_DIR, os.path.basename(src)[:-3] + ".o")
    cmd = ([nvcc()] + NVCC_FLAGS + (["-DDS_DEBUG_BOUNDS"] if bounds else []) +
           (["-Xptxas", "-v"] if verbose_ptxas else []) + ["-c", src, "-o", obj])
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def build(force=False, verbose_ptxas=False, jobs=None, bounds=False):
    """Compile (if stale) and return the path of libds.so (libds_bounds.so with
    bounds=True)."""
    lib, out_dir = (BOUNDS_LIB, BOUNDS_OUT_DIR) if bounds else (LIB, OUT_DIR)
    srcs = _sources()
    newest = max(os.path.getmtime(p) for p in srcs + _headers() + [__file__])
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest and not verbose_ptxas:
        return lib
    os.makedirs(out_dir, exist_ok=True)
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose_ptxas, bounds), srcs))
    if verbose_ptxas:
        for obj, log in results:
            sys.stderr.write(log)
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose_ptxas="-v" in sys.argv))
