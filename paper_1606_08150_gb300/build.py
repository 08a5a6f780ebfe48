"""Build the CUDA library libdpc.so (sm_103a, relocatable device code for CDP2).

Every translation unit is compiled in parallel with ``nvcc -dc`` and the objects
are device-linked into one shared library together with the device runtime
(``cudadevrt``), which device-side kernel launches need. Output goes next to
this file, inside the source tree.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdpc.so")
# the bounds-checked build (-DDPC_CHECKED): every index read from the caller's
# arrays and every append into a bounded buffer is checked on the device
CHECKED_FLAGS = ("-DDPC_CHECKED",)
LIB_CHECKED = os.path.join(HERE, "libdpc_checked.so")
BUILD_DIR_CHECKED = os.path.join(HERE, "_build_checked")
SOURCES = ["api.cu", "spmv.cu", "sssp.cu", "tree.cu", "rank.cu", "bfs.cu", "gc.cu", "noalloc.cu", "engine.cu", "diag.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdpc.so")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-rdc=true", "-Xcompiler", "-fPIC",
                   "-I", INCLUDE, "-I", CSRC, *extra]


def _needs_rebuild(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "dpc.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, extra_flags=(), checked: bool = False) -> str:
    """Compile libdpc.so (or, with checked=True, the bounds-checked
    libdpc_checked.so) if any source is newer than it; returns its path."""
    lib = LIB_CHECKED if checked else LIB
    build_dir = BUILD_DIR_CHECKED if checked else BUILD_DIR
    if checked:
        extra_flags = tuple(extra_flags) + CHECKED_FLAGS
    if not force and not _needs_rebuild(lib):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    flags = _flags(extra_flags)

    def compile_one(src):
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        cmd = [cc, *flags, "-dc", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-rdc=true", "-Xcompiler", "-fPIC", *objs, "-lcudadevrt", "-o", tmp]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
