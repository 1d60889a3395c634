"""Builds the CUDA library libhh.so in-tree for sm_103a (GB300).

Each source in csrc/ is compiled by nvcc in parallel into _build/, then linked
into paper_2603_02048_gb300/libhh.so against the shared CUDA runtime (the one
PyTorch also loads, so streams are interchangeable). The "debug_bounds"
variant (libhh_debug_bounds.so, compiled with -DHH_DEBUG_BOUNDS) checks every
trilinear corner index of the march against the padded volume; the tests
build it on demand. Usage:
    python -m paper_2603_02048_gb300.build [--variant debug_bounds]
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
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libhh.so")
VARIANTS = {None: ("libhh.so", "", ()), "debug_bounds": ("libhh_debug_bounds.so", "debug_bounds",
                                                        ("-DHH_DEBUG_BOUNDS",))}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    path = os.path.join(cuda, "bin", "nvcc")
    return path if os.path.exists(path) else (shutil.which("nvcc") or "nvcc")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _sources() + _headers() + [__file__])


def _compile(src: str, extra, build_dir: str) -> str:
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj, *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, extra=(), variant=None) -> str:
    """Compiles csrc/ into libhh.so (or the named variant's library) unless it
    is up to date; returns its path."""
    name, sub, defs = VARIANTS[variant]
    lib = os.path.join(PKG, name)
    if not force and not _stale(lib):
        return lib
    build_dir = os.path.join(BUILD, sub) if sub else BUILD
    os.makedirs(build_dir, exist_ok=True)
    srcs = _sources()
    flags = list(defs) + list(extra)
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, flags, build_dir), srcs))
    tmp = lib + ".tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print("built", lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else (),
          variant="debug_bounds" if "debug_bounds" in sys.argv else None)
