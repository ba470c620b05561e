"""Builds the in-tree CUDA library ``libradic.so`` for sm_103a with nvcc.

Each translation unit is compiled in parallel and the objects are linked into
one shared library next to this file (the CUDA runtime is linked statically,
so the library only needs the driver at run time).  Usage:
``python -m paper_1508_01326_gb300.build`` or ``build()`` from Python.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(HERE, "libradic.so")

SOURCES = [
    "radic_api.cu",
    "radic_fp64.cu",
    "radic_mixed.cu",
    "radic_pair.cu",
    "radic_modp.cu",
    "radic_modp_prefix.cu",
    "radic_noalloc.cu",
    "radic_batched.cu",
    "radic_batched_k32.cu",
    "radic_batched_kpair.cu",
    "radic_batched_k64.cu",
    "radic_backward.cu",
]

# The pipe-throughput probe whose measured peaks the bench's roofline
# fractions divide by: a measuring instrument, linked into its own library.
PEAK_SOURCES = ["radic_peaks.cu"]
PEAKS_LIB_PATH = os.path.join(HERE, "libradic_peaks.so")

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", f"-I{INCLUDE}", f"-I{CSRC}"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libradic.so")
    return cand


def _compile(src: str, verbose_ptxas: bool) -> str:
    obj = os.path.join(BUILD_DIR, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), *ARCH_FLAGS, *COMMON_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    if verbose_ptxas:
        with open(obj + ".ptxas.txt", "w") as f:
            f.write(res.stderr)
    return obj


def _stale() -> bool:
    if not os.path.exists(LIB_PATH) or not os.path.exists(PEAKS_LIB_PATH):
        return True
    lib_t = min(os.path.getmtime(LIB_PATH), os.path.getmtime(PEAKS_LIB_PATH))
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return any(os.path.getmtime(d) > lib_t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None) -> str:
    """Compiles every CUDA source for sm_103a and links libradic.so; returns its path."""
    if not force and not _stale():
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    jobs = jobs or min(len(SOURCES) + len(PEAK_SOURCES), os.cpu_count() or 4)
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas), SOURCES + PEAK_SOURCES))
    for path, lib_objs in ((LIB_PATH, objs[:len(SOURCES)]), (PEAKS_LIB_PATH, objs[len(SOURCES):])):
        tmp = path + ".tmp"
        cmd = [_nvcc(), *ARCH_FLAGS, "-shared", "-o", tmp, *lib_objs]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, path)
    return LIB_PATH


if __name__ == "__main__":
    path = build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv)
    print(path)
