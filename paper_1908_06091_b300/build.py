"""Build the library's CUDA/C++ sources into an in-tree shared object.

    python -m paper_1908_06091_b300.build      # or build() from Python
    python -m paper_1908_06091_b300.build debug

Compiles every ``csrc/*.cu`` and ``csrc/*.cpp`` with nvcc for sm_103a only
(``-gencode arch=compute_103a,code=sm_103a``) and links
``paper_1908_06091_b300/_lib/libnabla_b300.so``.  Objects go to ``_build/``.
A source is recompiled when it or any header in ``csrc/`` or ``include/``
is newer than its object.

The ``debug`` variant adds ``-DNB_BOUNDS_CHECK`` (kernels check every
gathered index against its buffer and record NB_EINVAL in the device status
word instead of reading outside it) and links
``_lib/libnabla_b300_debug.so`` from objects in ``_build/debug/``; the
binding loads it when ``NB_LIBRARY=debug`` is set.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libnabla_b300.so")
VARIANTS = {"": ([], OBJ, LIB),
            "debug": (["-DNB_BOUNDS_CHECK"], os.path.join(OBJ, "debug"),
                      os.path.join(LIBDIR, "libnabla_b300_debug.so"))}

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fopenmp,-O3",
          "-I" + os.path.join(ROOT, "include")]
CUFLAGS = ARCH + COMMON + ["--expt-relaxed-constexpr", "-Xptxas", "-O3"]


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    return max([os.path.getmtime(h) for h in hs] + [0.0])


def _compile(src: str, hdr_t: float, verbose: bool, extra=(), objdir: str = OBJ) -> str:
    obj = os.path.join(objdir, os.path.basename(src) + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_t):
        return obj
    flags = (CUFLAGS if src.endswith(".cu") else ARCH + COMMON) + list(extra)
    cmd = [NVCC] + flags + ["-c", src, "-o", obj + ".tmp"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, force: bool = False, variant: str = "") -> str:
    extra, objdir, lib = VARIANTS[variant]
    os.makedirs(objdir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr_t = _headers_mtime()
    if force:
        for o in glob.glob(os.path.join(objdir, "*.o")):
            os.remove(o)
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(lambda s: _compile(s, hdr_t, verbose, extra, objdir), srcs))
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < newest:
        cmd = [NVCC] + ARCH + ["-shared", "-o", lib + ".tmp"] + objs + \
            ["-Xcompiler", "-fopenmp", "-lgomp", "-lcudart"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    v = "debug" if "debug" in sys.argv else ""
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv, variant=v))
