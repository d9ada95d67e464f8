"""Build libbs.so in-tree from csrc/*.cu for sm_103a (nvcc, no cmake).

Every translation unit compiles in parallel to an object file, then nvcc
links the shared library.  Flags:
  -gencode arch=compute_103a,code=sm_103a   GB300 only
  --fmad=false                              no implicit contraction: every
                                            fused multiply-add is explicit
  -cudart shared                            share the process's CUDA runtime
Output: paper_2009_10917_gb300/_build/libbs.so; with --check (-DBS_CHECK=1,
device-side index checks) paper_2009_10917_gb300/_build_check/libbs.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libbs.so")
# the checked build (-DBS_CHECK=1: device-side index checks)
BUILD_CHECK = os.path.join(PKG, "_build_check")
LIB_CHECK = os.path.join(BUILD_CHECK, "libbs.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-Wall", "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [__file__])


# Sources of the seven BS kernels (BS1-BS7) and the device helpers they
# include (the C header holds declarations only): BS1-BS5, BS7, BS6.
STREAM_SOURCES = ("bs_internal.cuh", "bs_check.cuh", "bs_check_pred.h", "bs_stream.cuh",
                  "bs_stream.cu")
SCATTER_SOURCES = STREAM_SOURCES + ("bs_gs.cuh", "bs_gs.cu")
GATHER_SOURCES = SCATTER_SOURCES + ("bs_gather.cuh", "bs_tiles.h")
OP_SOURCES = {"copy": STREAM_SOURCES, "axpy": STREAM_SOURCES, "norm": STREAM_SOURCES,
              "dot": STREAM_SOURCES, "cg_update": STREAM_SOURCES, "scatter": SCATTER_SOURCES,
              "gather": GATHER_SOURCES}


def source_digest(names=None) -> str:
    """SHA-256 over the kernel sources and headers (identifies a build), or
    over the named files only (e.g. STREAM_SOURCES)."""
    import hashlib
    h = hashlib.sha256()
    for d in sorted(_deps()):
        if d == __file__ or (names is not None and os.path.basename(d) not in names):
            continue
        with open(d, "rb") as f:
            h.update(os.path.basename(d).encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def lib_path(check: bool = False) -> str:
    return LIB_CHECK if check else LIB


def is_stale(check: bool = False) -> bool:
    lib = lib_path(check)
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=None,
          check: bool = False) -> str:
    """Compile (if stale) and return the path of libbs.so; check=True builds
    the checked variant (-DBS_CHECK=1) into its own folder."""
    lib = lib_path(check)
    if not force and not is_stale(check):
        return lib
    out = BUILD_CHECK if check else BUILD
    os.makedirs(out, exist_ok=True)
    cc = nvcc()
    flags = NVCC_FLAGS + (["-DBS_CHECK=1"] if check else []) + list(extra_flags or [])
    objs = []

    def compile_one(src):
        obj = os.path.join(out, os.path.basename(src)[:-3] + ".o")
        cmd = [cc] + ARCH + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return obj

    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
        "-Xlinker", "-rpath=/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None,
                check="--check" in sys.argv))
