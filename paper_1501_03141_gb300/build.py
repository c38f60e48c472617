"""Build libpdep.so in-tree with nvcc for sm_103a.

Each translation unit of csrc/ is compiled in parallel and linked into
paper_1501_03141_gb300/libpdep.so.  Rebuilds only when a source or header is
newer than the library.  build(bounds_check=True) makes the debug variant
libpdep_check.so (-DPDEP_BOUNDS_CHECK: the transform kernels test every index
they read from the sphere tables), selected at import by PDEP_BOUNDS_CHECK=1.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpdep.so")
OUT_DIR_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(HERE, "libpdep_check.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "--extended-lambda", "-lineinfo", "-Xcompiler", "-fPIC",
         "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpdep.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, bounds_check: bool = False) -> str:
    """Compile every CUDA source for sm_103a and link libpdep.so (libpdep_check.so
    with bounds_check); returns its path."""
    lib = LIB_CHECK if bounds_check else LIB
    out_dir = OUT_DIR_CHECK if bounds_check else OUT_DIR
    flags = FLAGS + (["-DPDEP_BOUNDS_CHECK"] if bounds_check else [])
    if not force and not _stale(lib):
        return lib
    nvcc = _nvcc()
    os.makedirs(out_dir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, bounds_check="--bounds-check" in sys.argv[1:]))
