"""Wide exact mode (radic_det_exact_wide): det_R of Definition 3 / Eq. (1)
exactly, with as many 31-bit primes as the Hadamard bound of the scaled
integer rows needs (beyond the 128-bit result of radic_det's EXACT mode),
against the oracle's exact rational values."""
from fractions import Fraction

import numpy as np
import pytest

from conftest import read_golden_rows
from oracle import radic_oracle as orc
from paper_1508_01326_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def R():
    import paper_1508_01326_gb300 as mod

    return mod


def test_wide_fp64_8x32_equals_golden_fraction():
    # the 8 x 32 binary64 workload: the exact fraction written by the oracle
    # (Pfaffian closed form) into workload_exact.txt, bit for bit
    row = [r for r in read_golden_rows("workload_exact.txt") if r[0] == "fp64_8x32"][0]
    want = Fraction(int(row[2]), int(row[3]))
    res = R().det_exact_wide(W.fp64_8x32())
    assert res["value_exact"] == want
    assert res["n_primes"] > 4  # beyond radic_det's prime budget
    assert res["minors"] == 10518300
    assert abs(res["value"] - float(want)) <= 2.0 ** -51 * abs(float(want))
    # radic_det's EXACT mode cannot hold this value
    import torch

    a = torch.from_numpy(W.fp64_8x32()).cuda()
    r = R().parse_result(R().radic_det(a, mode="exact"))
    assert r["status"] == 2  # RADIC_EOVERFLOW


@pytest.mark.parametrize("m,n,seed,dtype", [(3, 7, 1, np.float64), (5, 11, 2, np.float64), (6, 13, 3, np.float64),
                                            (8, 16, 4, np.float64), (7, 14, 5, np.float32), (10, 15, 6, np.float64)])
def test_wide_real_inputs_match_oracle(m, n, seed, dtype):
    a = W.uniform_matrix(seed, m, n, dtype)
    want = orc.radic_det_pfaffian(a)
    for mapping in ("auto", "thread", "prefix"):
        if mapping == "thread" and m > 12:
            continue
        res = R().det_exact_wide(a, options={"mapping": mapping})
        assert res["value_exact"] == want, mapping


def test_wide_integer_beyond_int128_matches_oracle():
    # int32 entries near 2^30: det_R far beyond 2^127
    rng = np.random.default_rng(7)
    a = rng.integers(-(2 ** 30), 2 ** 30, (9, 13)).astype(np.int32)
    want = orc.radic_det_pfaffian(a)
    assert abs(want) > 2 ** 200
    res = R().det_exact_wide(a)
    assert res["value_exact"] == want and res["exact_exp"] == 0
    assert res["n_primes"] >= 8


def test_wide_agrees_with_exact_mode_where_it_fits():
    a = W.int8_10x24()
    res = R().det_exact_wide(a)
    ref = R().det(a, mode="exact")
    assert res["integer"] == ref["exact"] and res["n_primes"] == ref["n_primes"]


def test_wide_degenerate_cases():
    # m > n: det_R = 0 with no minors; a zero matrix; a rank-deficient one
    res = R().det_exact_wide(np.ones((5, 3)))
    assert res["integer"] == 0 and res["sign"] == 0 and res["minors"] == 0
    res = R().det_exact_wide(np.zeros((4, 9)))
    assert res["integer"] == 0 and res["sign"] == 0
    b = W.integer_matrix(9, 3, 8, 50).astype(np.float64)
    c = np.vstack([b, b[0] + b[1]])  # a row that is the sum of two others: every minor is 0
    res = R().det_exact_wide(c)
    assert res["value_exact"] == orc.radic_det_pfaffian(c) == 0


def test_wide_overflow_is_reported():
    # rows spanning about a thousand bits each: the bound needs far more
    # than RADIC_WIDE_MAX_PRIMES primes
    a = W.uniform_matrix(11, 6, 10)
    a[:, 0] = 1e-300
    with pytest.raises(R().RadicError):
        R().det_exact_wide(a)
