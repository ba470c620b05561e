"""Binary64 enumeration of Eq. (1) on the host cores (oracle/radic_cpu.c).

TEST AND MEASUREMENT INFRASTRUCTURE ONLY: loaded by tests/ and by the
CPU-baseline leg of bench.py, never by the library.  ``build()`` compiles the
C source with gcc and OpenMP into oracle/libradic_cpu.so (git-ignored);
``__graft_entry__.build()`` calls it so that the box has it before the tests.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "radic_cpu.c")
LIB = os.path.join(HERE, "libradic_cpu.so")
_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = shutil.which("gcc") or "cc"
    tmp = LIB + ".tmp"
    subprocess.run([cc, "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


def _load() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        L.radic_cpu_sum.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                    ctypes.c_uint64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
        L.radic_cpu_sum.restype = ctypes.c_double
        _lib = L
    return _lib


def radic_cpu_sum(a, q0: int = 0, count: int | None = None):
    """(sum, sum of magnitudes, threads used) of the signed minors with ranks q0 .. q0+count-1."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    m, n = a.shape
    if count is None:
        count = 2 ** 63
    ab = ctypes.c_double(0.0)
    th = ctypes.c_int(0)
    s = _load().radic_cpu_sum(a.ctypes.data, m, n, n, int(q0), int(count), ctypes.byref(ab), ctypes.byref(th))
    return float(s), float(ab.value), int(th.value)
