import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def golden_path(name):
    return os.path.join(ROOT, "tests", "golden", name)


def read_golden_rows(name):
    rows = []
    with open(golden_path(name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


def golden_abs_sums(name):
    """sum|terms| of a workload from workload_abs_sum.txt (written by make_abs_sums.py from oracle/ only),
    as a list indexed like the workload's matrices."""
    vals = {int(r[1]): float(r[2]) for r in read_golden_rows("workload_abs_sum.txt") if r[0] == name}
    return [vals[i] for i in range(len(vals))]


def golden_values(name):
    """Nearest binary64 of the exact det_R of a workload (workload_exact.txt, oracle Pfaffian closed form)."""
    vals = {int(r[1]): float(r[4]) for r in read_golden_rows("workload_exact.txt") if r[0] == name}
    return [vals[i] for i in range(len(vals))]
