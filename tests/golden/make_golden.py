"""Writes the exact reference values of the seeded workloads (calls only oracle/).

Values come from the Pfaffian minor-summation closed form of the oracle
(``radic_det_pfaffian``), which the oracle's own tests pin against
enumeration of Eq. (1) on small inputs.  Output: workload_exact.txt, one line
per value: ``name index numerator denominator float``.

Run from the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle.radic_oracle as orc  # noqa: E402
from paper_1508_01326_gb300 import workloads as W  # noqa: E402


def main() -> None:
    lines = [
        "# Exact det_R of the seeded workloads (oracle Pfaffian closed form; see make_golden.py).",
        "# name index numerator denominator nearest-binary64",
        "# (batched entries keep only the nearest binary64; '-' marks the omitted exact fraction)",
    ]

    def put(name, idx, val, keep_fraction=True):
        if keep_fraction:
            lines.append(f"{name} {idx} {val.numerator} {val.denominator} {float(val)!r}")
        else:
            lines.append(f"{name} {idx} - - {float(val)!r}")

    put("int_3x12", 0, orc.radic_det_pfaffian(W.int_3x12().astype(np.int64)))
    put("fp64_8x32", 0, orc.radic_det_pfaffian(W.fp64_8x32()))
    put("int8_10x24", 0, orc.radic_det_pfaffian(W.int8_10x24().astype(np.int64)))
    put("int8_12x40", 0, orc.radic_det_pfaffian(W.int8_12x40().astype(np.int64)))
    mats = W.batched_4096()
    for i, a in enumerate(mats):
        put("batched_4096_f64", i, orc.radic_det_pfaffian(a), keep_fraction=False)
    for i, a in enumerate(mats):
        put("batched_4096_f32", i, orc.radic_det_pfaffian(a.astype(np.float32)), keep_fraction=False)
    with open(os.path.join(HERE, "workload_exact.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
