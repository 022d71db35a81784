"""Builds liblbm_rd3q81.so in-tree for sm_103a (GB300) with plain nvcc.

Each translation unit compiles in its own nvcc process (in parallel); the objects are
linked into ``paper_2409_05114_gb300/liblbm_rd3q81.so`` against the shared CUDA runtime so
that the library and PyTorch use the same runtime instance and device contexts.
Usage: ``python -m paper_2409_05114_gb300.build_lib`` (or ``__graft_entry__.build()``).
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "liblbm_rd3q81.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "serve.cu", "lattice_tables.cu", "aux_kernels.cu", "sc_f64.cu", "sc_f32.cu", "sc_f16.cu", "sc_bf16.cu", "totals_noalloc.cu", "diagnostics.cu", "selftest.cu",
           "sc_aa_f64.cu", "sc_aa_f32.cu", "sc_aa_f16.cu", "sc_aa_bf16.cu"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm_rd3q81")
    return cand


def cuda_lib_dir(nv: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nv))), "lib64")


def compile_one(nv: str, src: str, verbose: bool) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nv, "-std=c++17", "-O3", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
           "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    if verbose:
        sys.stdout.write(f"== {src}\n{res.stderr}")
    return obj


def build(verbose: bool = False) -> str:
    nv = nvcc()
    os.makedirs(BUILD, exist_ok=True)
    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: compile_one(nv, s, verbose), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nv, "-shared", *ARCH, "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath," + cuda_lib_dir(nv)]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
