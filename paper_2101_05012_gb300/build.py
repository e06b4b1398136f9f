"""Build libabea.so in-tree (paper_2101_05012_gb300/_build/) with nvcc for sm_103a.

The translation units compile in parallel; the CUDA runtime is linked
statically so the library needs only the driver at run time.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libabea.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["abea_align.cu", "abea_prep.cu", "abea_api.cpp", "abea_noalloc.cu", "abea_server.cpp", "abea_scalings.cu", "abea_events.cu", "abea_eventalign.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _compile(src: str, extra) -> str:
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj, *extra]
    subprocess.run(cmd, check=True)
    return obj


def build(extra_flags=(), verbose_ptxas: bool = False) -> str:
    """Compile and link libabea.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra_flags) + (["-Xptxas", "-v"] if verbose_ptxas else [])
    with concurrent.futures.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    tmp = LIB + ".tmp"
    subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"], check=True)
    os.replace(tmp, LIB)
    return LIB


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    srcs = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(CSRC, "abea_internal.h"),
                                                        os.path.join(INCLUDE, "abea.h")]
    return all(os.path.getmtime(s) <= t for s in srcs)


if __name__ == "__main__":
    print(build(verbose_ptxas=True))
