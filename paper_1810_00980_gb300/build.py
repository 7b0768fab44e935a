"""Build libtmotif.so (CUDA, sm_103a) in-tree with nvcc.

Each .cu file under csrc/ compiles to an object in parallel, then the shared
library is linked; the same sources compiled with TM_CHECKED give the
bounds-checked libtmotif_checked.so.  Objects and the library land in
paper_1810_00980_gb300/_build/ (git-ignored)."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libtmotif.so")
LIB_CHECKED = os.path.join(BUILD, "libtmotif_checked.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "--expt-relaxed-constexpr", "-I", INCLUDE, *extra]


def _compile(src: str, extra, sub: str = "") -> str:
    obj = os.path.join(BUILD, sub, os.path.basename(src) + ".o")
    deps = [src, *glob.glob(os.path.join(CSRC, "*.cuh")), os.path.join(INCLUDE, "tm.h")]
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(d) for d in deps):
        return obj
    tmp = obj + f".{os.getpid()}.tmp.o"
    subprocess.check_call([nvcc(), *_flags(extra), "-c", src, "-o", tmp])
    os.replace(tmp, obj)
    return obj


def _link(lib: str, objs, force: bool):
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + f".{os.getpid()}.tmp"
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
                               "-Xlinker", "-rpath=/usr/local/cuda/lib64"])
        os.replace(tmp, lib)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Both libraries: libtmotif.so and the bounds-checked libtmotif_checked.so (TM_CHECKED),
    every translation unit of both compiled in parallel."""
    os.makedirs(os.path.join(BUILD, "checked"), exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    if force:
        for o in glob.glob(os.path.join(BUILD, "*.o")) + glob.glob(os.path.join(BUILD, "checked", "*.o")):
            os.remove(o)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    jobs = [(s, extra, "") for s in srcs] + [(s, ["-DTM_CHECKED"], "checked") for s in srcs]
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(lambda j: _compile(*j), jobs))
    _link(LIB, objs[:len(srcs)], force)
    _link(LIB_CHECKED, objs[len(srcs):], force)
    return LIB


if __name__ == "__main__":
    print(build())
