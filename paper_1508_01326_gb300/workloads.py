"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module draws random matrices and nothing else: it holds none of the
determinant arithmetic.  The paper has no datasets or experiments, so every
workload is synthetic, drawn with numpy's PCG64 generator from fixed seeds on
the host (the GPU sees the same bits after a copy).

Workloads (sizes follow the five benchmark configurations of this library):

* ``int_3x12``   -- one 3 x 12 int32 matrix, entries uniform in [-9, 9], seed 1.
* ``fp64_8x32``  -- one 8 x 32 float64 matrix, entries uniform in [-1, 1), seed 2.
* ``int8_12x40`` -- one 12 x 40 int8 matrix, entries uniform in [-3, 3], seed 3;
  its leading 10 x 24 block is the small exact case.
* ``batched_4096`` -- 4096 matrices, m uniform in {2..10}, n = m + uniform{1..20},
  entries N(0, 1), seed 4; a float32 copy casts the same draws.
* ``diff_256x6x28`` -- 256 matrices of 6 x 28, entries uniform in [-1, 1), seed 5.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np


def int_3x12() -> np.ndarray:
    return np.random.default_rng(1).integers(-9, 10, (3, 12)).astype(np.int32)


def fp64_8x32() -> np.ndarray:
    return np.random.default_rng(2).uniform(-1.0, 1.0, (8, 32))


def int8_12x40() -> np.ndarray:
    return np.random.default_rng(3).integers(-3, 4, (12, 40)).astype(np.int8)


def int8_10x24() -> np.ndarray:
    return np.ascontiguousarray(int8_12x40()[:10, :24])


def batched_4096(count: int = 4096) -> List[np.ndarray]:
    """List of float64 matrices of uneven shapes (m in 2..10, n - m in 1..20)."""
    rng = np.random.default_rng(4)
    ms = rng.integers(2, 11, count)
    ds = rng.integers(1, 21, count)
    return [rng.standard_normal((int(m), int(m + d))) for m, d in zip(ms, ds)]


def diff_256x6x28() -> np.ndarray:
    return np.random.default_rng(5).uniform(-1.0, 1.0, (256, 6, 28))


def uniform_matrix(seed: int, m: int, n: int, dtype=np.float64, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Small seeded real matrix for parity cases of arbitrary shape."""
    return np.random.default_rng(seed).uniform(lo, hi, (m, n)).astype(dtype)


def integer_matrix(seed: int, m: int, n: int, bound: int, dtype=np.int32) -> np.ndarray:
    """Small seeded integer matrix with entries uniform in [-bound, bound]."""
    return np.random.default_rng(seed).integers(-bound, bound + 1, (m, n)).astype(dtype)


def pack_batch(mats: List[np.ndarray], dtype=np.float64) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """Concatenate row-major matrices into one buffer.

    Returns (data, m, n, offset) where matrix b occupies
    data[offset[b] : offset[b] + m[b] * n[b]] with leading dimension n[b].
    """
    ms = np.array([a.shape[0] for a in mats], dtype=np.int32)
    ns = np.array([a.shape[1] for a in mats], dtype=np.int32)
    sizes = ms.astype(np.int64) * ns.astype(np.int64)
    offs = np.zeros(len(mats), dtype=np.int64)
    if len(mats) > 1:
        offs[1:] = np.cumsum(sizes)[:-1]
    data = np.concatenate([np.ascontiguousarray(a, dtype=dtype).ravel() for a in mats]) if mats else np.zeros(0, dtype)
    return data, ms, ns, offs
