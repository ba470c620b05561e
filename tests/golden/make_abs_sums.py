"""Writes sum|terms| of the seeded workloads (calls only oracle/).

sum|terms| = sum over all ascending column sequences J of |det(A[:, J])|, the
scale against which Eq. (1)'s floating-point results are judged.  The parity
tests divide errors by these values rather than by the magnitude sum the GPU
reports, and check the GPU's sum against them.

Sources, per line:
  exact    -- the exact oracle (``radic_terms_exact``: exact Bareiss minors of
              Eq. (1) over every dictionary rank), rounded to binary64;
  binary64 -- the oracle's binary64 host enumeration (``cpu_enum``: partial-
              pivot LU per minor, compensated sums), which the oracle tests pin
              to the exact values; only three digits of this scale matter.

Output: workload_abs_sum.txt, one line per value: ``name index abs_sum source``.
Run from the repository root:  python tests/golden/make_abs_sums.py
(about two minutes of the exact oracle on 8 cores and two of the binary64
enumeration for the 4096-matrix batch).
"""
from __future__ import annotations

import math
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def _exact_chunk(args):
    name, lo, hi = args
    sys.path.insert(0, ROOT)
    from fractions import Fraction

    import oracle.radic_oracle as orc
    from paper_1508_01326_gb300 import workloads as W

    a = {"fp64_8x32": W.fp64_8x32, "int8_10x24": lambda: W.int8_10x24().astype(np.int64),
         "int_3x12": lambda: W.int_3x12().astype(np.int64)}[name]()
    return sum((abs(t) for t in orc.radic_terms_exact(a, range(lo, hi))), Fraction(0))


def exact_abs_sum(pool, name: str, total: int, cores: int) -> float:
    per = -(-total // (8 * cores))
    chunks = [(name, lo, min(lo + per, total)) for lo in range(0, total, per)]
    return float(sum(pool.map(_exact_chunk, chunks)))


def main() -> None:
    from oracle import cpu_enum
    from paper_1508_01326_gb300 import workloads as W

    cores = os.cpu_count() or 1
    lines = ["# sum over J of |det(A[:, J])| of the seeded workloads (see make_abs_sums.py).",
             "# name index abs_sum source"]
    pool = mp.get_context("spawn").Pool(cores)
    try:
        for name, m, n in (("int_3x12", 3, 12), ("int8_10x24", 10, 24), ("fp64_8x32", 8, 32)):
            lines.append(f"{name} 0 {exact_abs_sum(pool, name, math.comb(n, m), cores)!r} exact")
    finally:
        pool.terminate()
    mats = W.batched_4096()
    for tag, cast in (("batched_4096_f64", np.float64), ("batched_4096_f32", np.float32)):
        for i, a in enumerate(mats):
            if a.shape[0] > a.shape[1]:
                s = 0.0
            else:
                _, s, _ = cpu_enum.radic_cpu_sum(a.astype(cast).astype(np.float64))
            lines.append(f"{tag} {i} {s!r} binary64")
    for i, a in enumerate(W.diff_256x6x28()):
        _, s, _ = cpu_enum.radic_cpu_sum(a)
        lines.append(f"diff_256x6x28 {i} {s!r} binary64")
    with open(os.path.join(HERE, "workload_abs_sum.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
