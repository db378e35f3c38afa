"""Build librgeo.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into a shared
library next to this file.  No cmake; the whole build takes well under a
minute.  The CUDA runtime is linked statically into the library.
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
BUILD = os.path.join(ROOT, "_build", "librgeo")
LIB = os.path.join(HERE, "librgeo.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (source, object name, extra flags): rgeo_trace.cu is compiled in three parts
SOURCES = [("rgeo_api.cu", "rgeo_api", []), ("rgeo_trace.cu", "rgeo_trace_p1", ["-DRGEO_TRACE_PART=1", "-diag-suppress=177"]),
           ("rgeo_trace.cu", "rgeo_trace_p2", ["-DRGEO_TRACE_PART=2", "-diag-suppress=177"]),
           ("rgeo_trace.cu", "rgeo_trace_p3", ["-DRGEO_TRACE_PART=3", "-diag-suppress=177"]), ("rgeo_noalloc.cu", "rgeo_noalloc", []),
           ("rgeo_mlp.cu", "rgeo_mlp", []), ("rgeo_scene_build.cpp", "rgeo_scene_build", [])]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librgeo")


def _compile(unit, extra=()) -> str:
    src, name, defs = unit
    obj = os.path.join(BUILD, name + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
           "-I", INCLUDE, "-I", CSRC, *defs, "-c", os.path.join(CSRC, src), "-o", obj, *extra]
    if src.endswith(".cpp"):
        cmd[cmd.index("-c")] = "-x=c++"
        cmd.insert(cmd.index("-x=c++") + 1, "-c")
    subprocess.check_call(cmd)
    return obj


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "rgeo.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose_ptxas="-v" in sys.argv))
