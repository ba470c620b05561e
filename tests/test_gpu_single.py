"""GPU parity of the single-matrix path against the exact oracle.

Element-by-element: the per-minor signed terms and the unranked column
sequences of the device are compared with the oracle for every rank of small
cases (several tasks and a ragged tail).  Whole results: det_R(A) against the
exact value, bit-exact for the multi-modular path, within
1e-12 * sum|terms| for binary64 and within derived bounds for the mixed
binary32 path and the pair (float-float) path.  Full-size workloads run in the launch configuration the bench
uses and are checked against the Pfaffian closed form and sampled terms.
"""
import itertools
import math
import random
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle.radic_oracle as orc
from paper_1508_01326_gb300 import workloads as W
from tests.conftest import golden_abs_sums

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
UPAIR = 2.0 ** -44  # unit roundoff allowed for the pair arithmetic (about 2^-46 per operation)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1508_01326_gb300 import build as B

    B.build()


def R():
    import paper_1508_01326_gb300 as R_

    return R_


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def hadamard_terms(a, combos):
    """Per-minor Hadamard bounds prod_i ||A[i, J]||_2 (tolerance scale)."""
    a = np.asarray(a, dtype=np.float64)
    j = np.asarray(combos, dtype=np.int64)
    sq = a[:, j] ** 2  # (m, count, m)
    return np.prod(np.sqrt(sq.sum(axis=2)), axis=0)


def combos0(n, m):
    return [tuple(c - 1 for c in cols) for cols in orc.lex_combinations(n, m)]


OPTS = {
    "thread": dict(mapping="thread"),
    "thread_l13": dict(mapping="thread", ranks_per_task=13, threads_per_block=64),
    "g16": dict(mapping="group", group_width=16),
    "g16_l5": dict(mapping="group", group_width=16, ranks_per_task=5),
    "g32": dict(mapping="group", group_width=32, ranks_per_task=7),
    "prefix": dict(mapping=3),
    "prefix_r1": dict(mapping=3, ranks_per_task=1, threads_per_block=64),
    "prefix2": dict(mapping=3, prefix_depth=2),
    "prefix3": dict(mapping=3, prefix_depth=3),
    "prefix3_r1": dict(mapping=3, prefix_depth=3, ranks_per_task=1, threads_per_block=64),
    # several lanes share the leaves of one prefix
    "prefix_lp4": dict(mapping=3, prefix_depth=2, lanes_per_prefix=4),
    "prefix3_lp8": dict(mapping=3, prefix_depth=3, lanes_per_prefix=8, ranks_per_task=1, threads_per_block=64),
    "prefix3_lp32": dict(mapping=3, prefix_depth=3, lanes_per_prefix=32),
}

_LP = ("prefix_lp4", "prefix3_lp8", "prefix3_lp32")
FP64_LIMIT = {"thread": 8, "thread_l13": 8, "prefix": 10, "prefix_r1": 10, "prefix2": 10, "prefix3": 10,
              "prefix3_r1": 10, **{k: 10 for k in _LP}}
MIXED_LIMIT = {"thread": 12, "thread_l13": 12, "prefix": 12, "prefix_r1": 12, "prefix2": 12, "prefix3": 12,
               "prefix3_r1": 12, **{k: 12 for k in _LP}}
PAIR_LIMIT = {"prefix": 10, "prefix_r1": 10, "prefix2": 10, "prefix3": 10, "prefix3_r1": 10, "thread": 0,
              **{k: 10 for k in _LP}}


# ---------------------------------------------------------------------------
# Unranking and successor (Section 4, Section 5)
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("n,m", [(8, 5), (10, 1), (10, 10), (12, 6), (13, 12), (16, 14), (18, 17), (20, 3)])
@pytest.mark.parametrize("L", [1, 7, 64])
def test_unrank_matches_dictionary_order(n, m, L):
    want = np.array(combos0(n, m), dtype=np.uint8)
    got = R().radic_unrank(n, m, 0, len(want), options=dict(ranks_per_task=L)).cpu().numpy()
    assert np.array_equal(got, want)


def test_unrank_table2():
    from tests.conftest import read_golden_rows

    rows = read_golden_rows("table2_lex_n8_m5.txt")
    want = np.array([[int(x) - 1 for x in r[1:]] for r in rows], dtype=np.uint8)
    got = R().radic_unrank(8, 5, 0, 56).cpu().numpy()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n,m", [(64, 32), (64, 1), (33, 32), (40, 12), (32, 8), (28, 6), (30, 20)])
def test_unrank_large_runs(n, m):
    total = math.comb(n, m)
    rng = random.Random(n * 100 + m)
    starts = {0, max(total - 150, 0)} | {rng.randrange(total) for _ in range(4)}
    for q0 in sorted(starts):
        count = min(150, total - q0)
        got = R().radic_unrank(n, m, q0, count, options=dict(ranks_per_task=11)).cpu().numpy()
        seq = orc.unrank_combinatorial_addition(q0, n, m)
        for r in range(count):
            assert list(got[r] + 1) == seq, (q0 + r)
            if r + 1 < count:
                seq = orc.lex_successor(seq, n)


# ---------------------------------------------------------------------------
# Per-minor terms, element by element
# ---------------------------------------------------------------------------

TERM_CASES = [
    # (m, n, dtype, options key)
    (1, 9, np.float64, "thread"),
    (3, 12, np.int32, "thread"),
    (5, 16, np.float64, "thread_l13"),
    (8, 14, np.float64, "thread"),
    (8, 13, np.float32, "thread_l13"),
    (6, 11, np.int8, "thread"),
    (10, 14, np.float64, "g16"),
    (12, 15, np.float64, "g16_l5"),
    (17, 19, np.float64, "g32"),
    (3, 9, np.float64, "prefix"),
    (4, 13, np.int32, "prefix_r1"),
    (5, 16, np.float64, "prefix"),
    (8, 14, np.float64, "prefix"),
    (8, 13, np.float32, "prefix_r1"),
    (10, 14, np.float64, "prefix"),
    (12, 15, np.float64, "prefix"),
    (4, 11, np.float64, "prefix3"),
    (5, 14, np.int32, "prefix3_r1"),
    (8, 14, np.float64, "prefix3"),
    (8, 13, np.float32, "prefix2"),
    (10, 15, np.float64, "prefix3"),
    (12, 16, np.float64, "prefix3"),
    (8, 14, np.float64, "prefix_lp4"),
    (8, 16, np.float64, "prefix3_lp8"),
    (6, 20, np.float32, "prefix3_lp32"),
    (10, 15, np.float64, "prefix3_lp32"),
]


def _matrix(m, n, dtype, seed):
    if np.dtype(dtype).kind == "i":
        return W.integer_matrix(seed, m, n, 3 if dtype == np.int8 else 9, dtype)
    return W.uniform_matrix(seed, m, n, dtype)


@pytest.mark.parametrize("m,n,dtype,key", TERM_CASES)
def test_terms_fp64_elementwise(m, n, dtype, key):
    if m > FP64_LIMIT.get(key, 32):
        pytest.skip("outside the binary64 limit of this mapping")
    a = _matrix(m, n, dtype, 100 + m * n)
    total = math.comb(n, m)
    q0 = total // 7
    count = total - q0
    got = R().radic_terms(dev(a), q0, count, mode="fp64", options=OPTS[key]).cpu().numpy()
    want = np.array([float(x) for x in orc.radic_terms_exact(a, range(q0, q0 + count))])
    h = hadamard_terms(a, combos0(n, m)[q0:])
    assert np.all(np.abs(got - want) <= 1e-13 * h + 1e-300), np.max(np.abs(got - want) / h)


# The growth rule of the mixed mode, restated in binary64 on the host (test
# logic, not the oracle): rows are scaled by powers of two so that each row's
# largest entry lies in [0.5, 1); a per-minor LU flags its minor when its
# largest pivot exceeds the threshold; a prefix flags all minors of its
# subtree when its largest pivot, or 2^(D-1) times the largest Schur-complement
# entry of its candidate columns, exceeds the threshold.
GROWTH_THR = 64.0


def _scaled_rows(a):
    a = np.asarray(a, dtype=np.float64)
    mx = np.abs(a).max(axis=1)
    e = np.where(mx > 0, np.frexp(mx)[1], 0)
    return np.ldexp(a, -e[:, None])


def _eliminate(stack, steps):
    """Partial-pivot elimination of the first `steps` columns of a stack (N, m, c), pivot rows
    chosen among the not yet eliminated rows; returns the pivots (N, steps) and the reduced stack."""
    s = np.array(stack, dtype=np.float64, copy=True)
    N = s.shape[0]
    piv = np.zeros((N, steps))
    idx = np.arange(N)
    for k in range(steps):
        p = k + np.argmax(np.abs(s[:, k:, k]), axis=1)
        rk = s[idx, k, :].copy()
        s[idx, k, :] = s[idx, p, :]
        s[idx, p, :] = rk
        piv[:, k] = s[:, k, k]
        with np.errstate(divide="ignore", invalid="ignore"):
            l = s[:, k + 1:, k] / s[:, k, k][:, None]
        l = np.where(np.isfinite(l), l, 0.0)
        s[:, k + 1:, k:] -= l[:, :, None] * s[:, k, None, k:]
    return piv, s


def mixed_growth_rule(a, m, n, depth):
    """Per dictionary rank, the quantity the mixed mode compares with its threshold, and the
    smallest pivot magnitude that divides (per-minor: all pivots but the last; prefix: the
    prefix pivots), whose binary32 enclosure may reach zero and also flag the minor."""
    s = _scaled_rows(a)
    combos = combos0(n, m)
    if depth == 0:  # per-minor LU
        piv, _ = _eliminate(np.stack([s[:, list(c)] for c in combos]), m)
        minpiv = np.abs(piv[:, :-1]).min(axis=1) if m > 1 else np.full(len(combos), np.inf)
        return np.abs(piv).max(axis=1), minpiv
    P = m - depth
    rule_of_prefix, min_of_prefix = {}, {}
    for v in range(P - 1, n - depth):
        heads = list(itertools.combinations(range(v), P - 1))
        cand = list(range(v + 1, n))
        stack = np.stack([np.concatenate([s[:, list(h) + [v]], s[:, cand]], axis=1) for h in heads])
        piv, red = _eliminate(stack, P)
        zmax = np.abs(red[:, P:, P:]).max(axis=(1, 2))
        r = np.maximum(np.abs(piv).max(axis=1), 2.0 ** (depth - 1) * zmax)
        for h, val, mp in zip(heads, r, np.abs(piv).min(axis=1)):
            rule_of_prefix[h + (v,)] = val
            min_of_prefix[h + (v,)] = mp
    return (np.array([rule_of_prefix[c[:P]] for c in combos]), np.array([min_of_prefix[c[:P]] for c in combos]))


def _wilkinson_matrix(m, n, seed):
    # partial pivoting grows the last column of the leading minor to 2^(m-1)
    # times its entries (Wilkinson's example)
    w = np.eye(m) - np.tril(np.ones((m, m)), -1)
    w[:, -1] = 1.0
    return np.concatenate([w, W.uniform_matrix(seed, m, n - m)], axis=1)


MIXED_FLAG_CASES = TERM_CASES + [
    (9, 12, "wilkinson", "thread"),
    (9, 12, "wilkinson", "g16"),
    (9, 12, "wilkinson", "prefix2"),
    (9, 12, "wilkinson", "prefix3"),
    (9, 13, "wilkinson", "prefix3_lp8"),
]


@pytest.mark.parametrize("m,n,dtype,key", MIXED_FLAG_CASES)
def test_terms_mixed_elementwise(m, n, dtype, key):
    if m > MIXED_LIMIT.get(key, 32):
        pytest.skip("outside the binary32 limit of this mapping")
    a = _wilkinson_matrix(m, n, 8) if dtype == "wilkinson" else _matrix(m, n, dtype, 200 + m * n)
    total = math.comb(n, m)
    q0 = total // 5
    count = total - q0
    got = R().radic_terms(dev(a), q0, count, mode="mixed", options=OPTS[key]).cpu().numpy()
    want = np.array([float(x) for x in orc.radic_terms_exact(a, range(q0, q0 + count))])
    h = hadamard_terms(a, combos0(n, m)[q0:])
    plan = R().radic_plan_info(m, n, "mixed", OPTS[key])
    rule, minpiv = mixed_growth_rule(a, m, n, plan["prefix_depth"] if plan["mapping"] == "prefix" else 0)
    # the NaN terms are exactly the minors the growth rule flags, outside a
    # band of 2^-10 around the threshold where the binary32 and binary64
    # values of the compared quantity may fall on different sides
    # (a quantity exactly at the threshold comes from exact arithmetic on
    # small integers, the same in both precisions, and is not flagged)
    band = (np.abs(rule - GROWTH_THR) <= GROWTH_THR * 2.0 ** -10) & (rule != GROWTH_THR)
    assert band.sum() <= max(2, len(band) // 1000)
    flagged = rule > GROWTH_THR
    nan = np.isnan(got)
    clear = ~band[q0:]
    # every minor the growth rule flags is NaN; the others that are NaN had a
    # dividing pivot so small that its binary32 enclosure reached zero (the
    # error bound's condition), and are few
    assert np.all(nan[clear] >= flagged[q0:][clear]), (nan.sum(), flagged[q0:].sum())
    extra = nan & ~flagged[q0:]
    assert extra.sum() <= max(2, len(extra) // 100), extra.sum()
    assert np.all(minpiv[q0:][extra] <= 1e-3), minpiv[q0:][extra]
    if dtype == "wilkinson":
        assert flagged.any()
    ok = ~nan
    # binary32 LU: backward error O(m u) per entry, plus the binary32 cast of binary64 input
    assert np.all(np.abs(got[ok] - want[ok]) <= 8 * m * U32 * h[ok]), np.max(np.abs(got[ok] - want[ok]) / h[ok])
    # the flagged minors through the binary64 path: their binary64 terms, and
    # the mixed determinant that recomputes them in binary64
    if nan.any():
        t64 = R().radic_terms(dev(a), q0, count, mode="fp64",
                              options=OPTS[key] if key.startswith("prefix") or m <= 8 else OPTS["g16"])
        t64 = t64.cpu().numpy()
        assert np.all(np.abs(t64[nan] - want[nan]) <= 1e-13 * h[nan])
    res = R().det(a, mode="mixed", options=OPTS[key])
    if not band.any():
        assert res["flagged"] >= int(flagged.sum())
    h_all = hadamard_terms(a, combos0(n, m))
    val, _ = _exact(a)
    assert_bounded(res, val)
    sure = flagged & ~band  # recomputed in binary64 whichever side the band minors fell
    bound = 8 * m * U32 * h_all[~sure].sum() + 1e-13 * h_all[sure].sum()
    assert abs(res["value"] - float(val)) <= bound


@pytest.mark.parametrize("m,n,dtype,key", TERM_CASES)
def test_terms_pair_elementwise(m, n, dtype, key):
    if not key.startswith("prefix") or m > PAIR_LIMIT[key]:
        pytest.skip("the pair mode has the prefix mapping only, m <= 10")
    a = _matrix(m, n, dtype, 250 + m * n)
    total = math.comb(n, m)
    q0 = total // 6
    count = total - q0
    got = R().radic_terms(dev(a), q0, count, mode="pair", options=OPTS[key]).cpu().numpy()
    want = np.array([float(x) for x in orc.radic_terms_exact(a, range(q0, q0 + count))])
    h = hadamard_terms(a, combos0(n, m)[q0:])
    # pair LU: backward error O(m u) per entry with u about 2^-46, and the
    # 48-bit rounding of binary64 input
    assert np.all(np.abs(got - want) <= 8 * m * UPAIR * h + 1e-300), np.max(np.abs(got - want) / h)


EXACT_CASES = [
    (1, 7, np.int32, "thread", 50),
    (3, 12, np.int32, "thread", 9),
    (4, 10, np.int8, "thread", 1),  # many zeros: zero pivots, singular minors
    (7, 12, np.int8, "thread_l13", 3),
    (12, 14, np.int8, "thread", 3),
    (9, 13, np.int32, "thread", 1000),
    (13, 16, np.int8, "g16", 3),
    (14, 15, np.int32, "g16_l5", 20),
    (18, 19, np.int8, "g32", 2),
    # prefix mapping in modular arithmetic (non-dividing elimination)
    (3, 12, np.int32, "prefix", 9),
    (4, 10, np.int8, "prefix", 1),  # many zeros: prefixes singular mod p
    (7, 12, np.int8, "prefix3", 3),
    (8, 14, np.int32, "prefix3", 1000),
    (6, 16, np.int8, "prefix_lp4", 3),
    (9, 16, np.int8, "prefix3_lp8", 3),
    (10, 15, np.int32, "prefix3_lp32", 50),
    (12, 15, np.int8, "prefix3", 3),
    (12, 16, np.int8, "prefix2", 2),
]


@pytest.mark.parametrize("m,n,dtype,key,bound", EXACT_CASES)
def test_terms_exact_elementwise(m, n, dtype, key, bound):
    a = W.integer_matrix(300 + m * n, m, n, bound, dtype)
    total = math.comb(n, m)
    q0 = total // 3
    count = total - q0
    out = R().radic_terms(dev(a), q0, count, mode="exact", options=OPTS[key]).cpu().numpy().view(np.uint32)
    res = R().det(a, mode="exact", options=OPTS[key])
    k_used = res["n_primes"]
    primes = R().radic_primes()
    want = orc.radic_terms_exact(a.astype(np.int64), range(q0, q0 + count))
    for k in range(k_used):
        p = primes[k]
        assert [int(x) for x in out[k, :count]] == [int(w) % p for w in want], k


# ---------------------------------------------------------------------------
# Whole determinants on small cases
# ---------------------------------------------------------------------------

DET_CASES = [
    (1, 1, np.float64), (1, 11, np.float64), (2, 3, np.float32), (3, 12, np.int32), (4, 4, np.float64),
    (5, 9, np.int8), (6, 13, np.float64), (7, 12, np.float32), (8, 8, np.float64), (8, 15, np.float64),
    (9, 13, np.float64), (10, 14, np.float32), (12, 16, np.float64), (16, 18, np.float64),
    (20, 22, np.float64), (3, 2, np.float64),
]


def _exact(a):
    return orc.radic_det_exact(a)


def assert_bounded(res, exact):
    """The result's err_bound is an upper bound on its actual error against the exact value."""
    err = abs(Fraction(res["value"]) - Fraction(exact))
    assert err <= Fraction(res["err_bound"]), (float(err), res["err_bound"])


def _mapping_ok(mapping, m, n, limits):
    if mapping == "auto":
        return True
    if mapping == "group":
        return m <= 32
    if mapping == "prefix":
        return 3 <= m <= limits["prefix"] and m <= n
    if mapping in ("prefix3", "prefix3_lp32"):
        return 4 <= m <= limits["prefix"] and m <= n
    return m <= limits["thread"]


def _det_opts(mapping):
    if mapping == "prefix3_lp32":
        return dict(OPTS[mapping])
    return dict(mapping=3, prefix_depth=3) if mapping == "prefix3" else dict(mapping=mapping)


@pytest.mark.parametrize("mapping", ["auto", "thread", "group", "prefix", "prefix3", "prefix3_lp32"])
@pytest.mark.parametrize("m,n,dtype", DET_CASES)
def test_det_fp64_small(m, n, dtype, mapping):
    if not _mapping_ok(mapping, m, n, FP64_LIMIT):
        pytest.skip("mapping does not cover this shape")
    a = _matrix(m, n, dtype, 400 + m * n)
    val, abs_sum = _exact(a)
    res = R().det(a, mode="fp64", options=_det_opts(mapping))
    assert res["minors"] == (math.comb(n, m) if m <= n else 0)
    assert abs(Fraction(res["value"]) - val) <= Fraction(1e-12) * abs_sum
    assert_bounded(res, val)
    if abs_sum:
        assert abs(res["abs_sum"] - float(abs_sum)) <= 1e-12 * float(abs_sum)
        assert res["err_bound"] <= 1e-8 * float(abs_sum)


@pytest.mark.parametrize("mapping", ["auto", "thread", "group", "prefix", "prefix3", "prefix3_lp32"])
@pytest.mark.parametrize("m,n,dtype", DET_CASES)
def test_det_mixed_small(m, n, dtype, mapping):
    if not _mapping_ok(mapping, m, n, MIXED_LIMIT):
        pytest.skip("mapping does not cover this shape")
    a = _matrix(m, n, dtype, 500 + m * n)
    val, abs_sum = _exact(a)
    res = R().det(a, mode="mixed", options=_det_opts(mapping))
    if m > n:
        assert res["value"] == 0.0 and res["minors"] == 0
        return
    h = hadamard_terms(a, combos0(n, m)).sum()
    assert abs(res["value"] - float(val)) <= 8 * m * U32 * h
    assert res["tier"] == 1
    assert_bounded(res, val)
    assert res["err_bound"] <= 2.0 ** -10 * h


@pytest.mark.parametrize("mapping", ["auto", "prefix", "prefix3", "prefix3_lp32"])
@pytest.mark.parametrize("m,n,dtype", DET_CASES)
def test_det_pair_small(m, n, dtype, mapping):
    if not (3 <= m <= 10 and m <= n and _mapping_ok(mapping, m, n, PAIR_LIMIT)):
        pytest.skip("the pair mode has the prefix mapping only, 3 <= m <= min(n, 10)")
    a = _matrix(m, n, dtype, 550 + m * n)
    val, abs_sum = _exact(a)
    res = R().det(a, mode="pair", options=_det_opts(mapping))
    assert res["tier"] == 3
    assert res["minors"] == math.comb(n, m)
    h = hadamard_terms(a, combos0(n, m)).sum()
    assert abs(res["value"] - float(val)) <= 8 * m * UPAIR * h
    assert abs(float(Fraction(res["value"]) - val)) <= 1e-11 * float(abs_sum)
    assert_bounded(res, val)
    assert res["err_bound"] <= 1e-10 * float(abs_sum)


def test_pair_mode_rejects_other_mappings_and_shapes():
    from paper_1508_01326_gb300 import RadicError

    with pytest.raises(RadicError):
        R().det(W.uniform_matrix(1, 5, 9), mode="pair", options=dict(mapping="thread"))
    with pytest.raises(RadicError):
        R().det(W.uniform_matrix(1, 11, 14), mode="pair")
    with pytest.raises(RadicError):
        R().det(W.uniform_matrix(1, 2, 14), mode="pair")


@pytest.mark.parametrize("mapping", ["auto", "thread"])
@pytest.mark.parametrize("m,n,dtype,bound", [(1, 5, np.int32, 7), (3, 12, np.int32, 9), (5, 9, np.int8, 3),
                                             (8, 11, np.int32, 3000), (10, 13, np.int8, 3),
                                             (12, 13, np.int32, 100), (13, 15, np.int8, 3),
                                             (16, 17, np.int32, 10), (4, 3, np.int8, 3), (7, 19, np.int8, 1)])
def test_det_exact_small(m, n, dtype, bound, mapping):
    if mapping == "thread" and m > 12:
        pytest.skip("thread mapping of the exact mode: m <= 12")
    a = W.integer_matrix(600 + m * n, m, n, bound, dtype)
    val, _ = _exact(a.astype(np.int64))
    res = R().det(a, mode="exact", options=dict(mapping=mapping))
    assert res["status"] == 0
    assert res["exact"] == val
    assert res["value"] == float(val)


def _dyadic(seed, m, n, dtype):
    # small integers times per-entry and per-row powers of two: binary32 and
    # binary64 hold them exactly, and the scaled integer rows stay short
    rng = np.random.default_rng(seed)
    k = rng.integers(-60, 61, (m, n))
    s = rng.integers(0, 5, (m, n))
    r = rng.integers(-6, 7, (m, 1))
    return (k * np.ldexp(1.0, -s) * np.ldexp(1.0, r)).astype(dtype)


@pytest.mark.parametrize("key", ["auto", "thread", "g16", "prefix2", "prefix3", "prefix3_lp8"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("m,n", [(1, 6), (3, 12), (6, 14), (8, 13)])
def test_det_exact_real_inputs(m, n, dtype, key):
    # Exact mode on real inputs: the integer matrix of the row-scaled entries
    # times 2^exact_exp, against the oracle's rational value
    if key.startswith("prefix") and m <= OPTS[key]["prefix_depth"]:
        pytest.skip("prefix mapping: m > prefix depth")
    a = _dyadic(700 + m * n, m, n, dtype)
    val, _ = orc.radic_det_exact(a.astype(np.float64))
    res = R().det(a, mode="exact", options=None if key == "auto" else OPTS[key])
    assert res["status"] == 0
    assert res["value_exact"] == val
    assert res["value"] == float(val)


def test_det_exact_real_inputs_limits():
    # random binary64 entries carry ~53 significant bits per entry: beyond
    # the prime budget, reported as RADIC_EOVERFLOW; a non-finite entry is
    # RADIC_EINVAL on the device
    out = R().radic_det(dev(W.uniform_matrix(5, 6, 12)), mode="exact")
    assert R().parse_result(out)["status"] == 2
    a = _dyadic(5, 4, 9, np.float64)
    a[2, 3] = np.inf
    out = R().radic_det(dev(a), mode="exact")
    assert R().parse_result(out)["status"] == 1
    # an all-zero row: every minor is zero
    a = _dyadic(6, 4, 9, np.float64)
    a[1] = 0.0
    res = R().parse_result(R().radic_det(dev(a), mode="exact"))
    assert res["status"] == 0 and res["exact"] == 0


def test_det_square_and_row_special_cases():
    rng = np.random.default_rng(9)
    for size in [1, 2, 5, 8]:
        a = rng.uniform(-1, 1, (size, size))
        assert abs(R().det(a)["value"] - np.linalg.det(a)) <= 1e-13 * max(1.0, abs(np.linalg.det(a)))
    row = np.array([[3, 1, 4, 1, 5]], dtype=np.int32)
    assert R().det(row, mode="exact")["exact"] == 10
    assert R().det(row.astype(np.float64))["value"] == 10.0


def test_det_leading_dimension():
    a = W.uniform_matrix(77, 6, 15)
    wide = np.zeros((6, 21))
    wide[:, :15] = a
    t = dev(wide)[:, :15]
    assert t.stride(0) == 21
    out = R().radic_det(t, mode="fp64")
    ref = R().det(a, mode="fp64")
    assert R().parse_result(out)["value"] == ref["value"]


def test_det_is_deterministic():
    # deterministic plans give the same bits on every call; the default prefix
    # schedule (tasks drawn from a counter) may change the rounding of the
    # sums only (the pair tier's lane totals are pair sums)
    a = dev(W.uniform_matrix(3, 7, 20))
    _, abs_sum = orc.radic_det_exact(W.uniform_matrix(3, 7, 20))
    for mode in ["fp64", "mixed", "pair"]:
        r1, r2 = (R().parse_result(R().radic_det(a, mode=mode, options=dict(deterministic=True))) for _ in range(2))
        assert (r1["value"], r1["abs_sum"], r1["err_bound"]) == (r2["value"], r2["abs_sum"], r2["err_bound"])
        d1, d2 = (R().parse_result(R().radic_det(a, mode=mode))["value"] for _ in range(2))
        assert abs(d1 - d2) <= 1e-13 * float(abs_sum)


@pytest.mark.parametrize("mode", ["fp64", "mixed", "pair"])
def test_prefix_task_schedules(mode):
    # 8 x 32: more warp tasks than warps.  A fixed task share per warp
    # (deterministic) gives the same bits on every call; tasks drawn from the
    # counter (default) change only the rounding of the sums.
    a = dev(W.fp64_8x32())
    fixed = [R().parse_result(R().radic_det(a, mode=mode, options=dict(deterministic=True))) for _ in range(3)]
    for r in fixed[1:]:
        assert (r["value"], r["abs_sum"]) == (fixed[0]["value"], fixed[0]["abs_sum"])
    for _ in range(3):
        r = R().parse_result(R().radic_det(a, mode=mode))
        assert abs(r["value"] - fixed[0]["value"]) <= 1e-13 * ABS_8X32
        assert abs(r["abs_sum"] - fixed[0]["abs_sum"]) <= 1e-13 * ABS_8X32


@pytest.mark.parametrize("key", ["thread", "g16", "prefix2", "prefix3", "prefix3_lp8", "prefix3_lp32"])
def test_mixed_growth_flag_recomputes_in_binary64(key):
    # Partial pivoting grows the last column of this minor to 2^(m-1) times
    # its entries (Wilkinson's example), above the default threshold 64.
    m, n = 9, 11
    w = np.eye(m) - np.tril(np.ones((m, m)), -1)
    w[:, -1] = 1.0
    a = np.concatenate([w, W.uniform_matrix(8, m, n - m)], axis=1)
    val, abs_sum = _exact(a)
    res = R().det(a, mode="mixed", options=OPTS[key])
    assert res["flagged"] >= 1
    h = hadamard_terms(a, combos0(n, m)).sum()
    assert abs(res["value"] - float(val)) <= 8 * m * U32 * h
    assert_bounded(res, val)


@pytest.mark.parametrize("key", ["prefix2", "prefix3", "prefix3_lp8"])
def test_pair_growth_flag_recomputes_in_binary64(key):
    m, n = 9, 11
    w = np.eye(m) - np.tril(np.ones((m, m)), -1)
    w[:, -1] = 1.0
    a = np.concatenate([w, W.uniform_matrix(18, m, n - m)], axis=1)
    val, abs_sum = _exact(a)
    res = R().det(a, mode="pair", options=OPTS[key])
    assert res["flagged"] >= 1
    h = hadamard_terms(a, combos0(n, m)).sum()
    assert abs(res["value"] - float(val)) <= 8 * m * UPAIR * h
    assert_bounded(res, val)


@pytest.mark.parametrize("mapping", ["thread", "prefix", "prefix3"])
def test_mixed_flag_list_overflow_falls_back_to_binary64(mapping):
    a = W.uniform_matrix(12, 6, 14)
    val, abs_sum = _exact(a)
    opts = _det_opts(mapping)
    opts.update(flag_capacity=1, growth_threshold=1e-30)
    res = R().det(a, mode="mixed", options=opts)
    assert res["flagged"] == math.comb(14, 6)
    assert abs(res["value"] - float(val)) <= 1e-12 * float(abs_sum)
    assert_bounded(res, val)


def test_exact_overflow_status():
    a = W.integer_matrix(5, 12, 14, 2 ** 30, np.int32)
    from paper_1508_01326_gb300 import RadicError

    with pytest.raises(RadicError) as e:
        R().det(a, mode="exact")
    assert e.value.code == 2


def test_workspace_too_small():
    from paper_1508_01326_gb300 import RadicError

    a = dev(W.uniform_matrix(1, 4, 9))
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(RadicError) as e:
        R().radic_det(a, workspace=ws)
    assert e.value.code == 5


# ---------------------------------------------------------------------------
# Full-size workloads (bench launch configuration)
# ---------------------------------------------------------------------------


def test_full_int_3x12_exact_and_fp64():
    a = W.int_3x12()
    val, abs_sum = orc.radic_det_exact(a.astype(np.int64))
    assert R().det(a, mode="exact")["exact"] == val
    res = R().det(a, mode="fp64")
    assert abs(Fraction(res["value"]) - val) <= Fraction(1e-12) * abs_sum
    h = hadamard_terms(a, combos0(12, 3)).sum()
    assert abs(R().det(a, mode="mixed")["value"] - float(val)) <= 8 * 3 * U32 * h


@pytest.fixture(scope="module")
def fp64_8x32():
    a = W.fp64_8x32()
    return a, orc.radic_det_pfaffian(a)


# Tolerance scale of the full-size tests: sum|terms| of the oracle (exact
# Bareiss minors over all 10,518,300 ranks, tests/golden/workload_abs_sum.txt),
# never the magnitude sum the GPU reports; the GPU's sum is itself checked
# against it (binary64 and pair sums to 1e-9, binary32-elimination sums to 1e-5:
# each |term| carries its minor's rounding, at most 8 m u of its Hadamard bound).
ABS_8X32 = golden_abs_sums("fp64_8x32")[0]


@pytest.mark.parametrize("mapping", ["auto", "thread", "prefix", "prefix3"])
def test_full_fp64_8x32_binary64(fp64_8x32, mapping):
    a, exact = fp64_8x32
    res = R().det(a, mode="fp64", options=_det_opts(mapping))
    assert res["minors"] == 10_518_300
    assert abs(Fraction(res["value"]) - exact) <= Fraction(1e-12) * Fraction(ABS_8X32)
    assert abs(res["abs_sum"] - ABS_8X32) <= 1e-9 * ABS_8X32
    # the a-posteriori bound holds and states the binary64 target
    assert_bounded(res, exact)
    assert res["err_bound"] <= 1e-12 * ABS_8X32


@pytest.mark.parametrize("mapping", ["auto", "thread"])
def test_full_fp64_8x32_mixed(fp64_8x32, mapping):
    a, exact = fp64_8x32
    res = R().det(a, mode="mixed", options=_det_opts(mapping))
    rel = abs(float(Fraction(res["value"]) - exact)) / ABS_8X32
    assert rel <= 1e-10, rel
    assert abs(res["abs_sum"] - ABS_8X32) <= 1e-5 * ABS_8X32
    # binary32 elimination: the bound holds, at the binary32 level
    assert_bounded(res, exact)
    assert res["err_bound"] <= 1e-3 * ABS_8X32


@pytest.mark.parametrize("mapping", ["auto", "prefix", "prefix3"])
def test_full_fp64_8x32_pair(fp64_8x32, mapping):
    a, exact = fp64_8x32
    res = R().det(a, mode="pair", options=_det_opts(mapping))
    assert res["tier"] == 3 and res["minors"] == 10_518_300
    rel = abs(float(Fraction(res["value"]) - exact)) / ABS_8X32
    assert rel <= 1e-12, rel
    assert abs(res["abs_sum"] - ABS_8X32) <= 1e-5 * ABS_8X32
    assert_bounded(res, exact)
    assert res["err_bound"] <= 1e-10 * ABS_8X32


def test_full_fp64_8x32_sampled_terms(fp64_8x32):
    a, _ = fp64_8x32
    rng = random.Random(22)
    t = dev(a)
    all_combos = None
    for _ in range(6):
        q0 = rng.randrange(10_518_300 - 300)
        got = R().radic_terms(t, q0, 300, mode="fp64").cpu().numpy()
        want = np.array([float(x) for x in orc.radic_terms_exact(a, range(q0, q0 + 300))])
        cols = [np.array(orc.unrank_combinatorial_addition(q, 32, 8)) - 1 for q in range(q0, q0 + 300)]
        h = hadamard_terms(a, cols)
        assert np.all(np.abs(got - want) <= 1e-13 * h)


def _paired_columns(m, half, eps, seed):
    """m x 2*half matrix whose columns come in adjacent pairs (b_i, b_i + eps d_i).

    Swapping the copy of one pair in a column sequence changes s by one and
    leaves the minor unchanged when eps = 0, so every term of Eq. (1) meets
    one of opposite sign and det_R(A) = 0 exactly; with eps > 0 the signed
    copies of each pair combine to -eps d_i, so the sum is of order
    eps^m * sum|terms| (2e-8 of it at eps = 1/4, m = 8).  The partners of a term whose first columns differ
    lie far apart in dictionary order, in different lanes and blocks, so the
    cancellation happens in the cross-lane and cross-block reductions.
    """
    rng = np.random.default_rng(seed)
    b = rng.uniform(-1.0, 1.0, (m, half))
    d = rng.uniform(-1.0, 1.0, (m, half))
    a = np.empty((m, 2 * half))
    a[:, 0::2] = b
    a[:, 1::2] = b + eps * d
    return a


@pytest.mark.parametrize("eps", [0.0, 2.0 ** -20, 0.25])
@pytest.mark.parametrize("mode,tol", [("fp64", 1e-12), ("mixed", 1e-10), ("pair", 1e-12)])
def test_cancelling_sums_across_lanes_and_blocks(mode, tol, eps):
    from oracle import cpu_enum

    a = _paired_columns(8, 16, eps, 77)
    exact = orc.radic_det_pfaffian(a)
    _, abs_sum, _ = cpu_enum.radic_cpu_sum(a)
    assert abs(float(exact)) <= 1e-4 * abs_sum  # the terms cancel to far below their magnitudes
    for opts in (None, dict(deterministic=True)):
        res = R().det(a, mode=mode, options=opts)
        assert abs(float(Fraction(res["value"]) - exact)) <= tol * abs_sum, (res, float(exact), abs_sum)
        assert_bounded(res, exact)


@pytest.mark.parametrize("mapping", ["auto", "thread", "prefix2"])
def test_full_int8_10x24_exact(mapping):
    a = W.int8_10x24()
    exact = orc.radic_det_pfaffian(a.astype(np.int64))
    opts = OPTS[mapping] if mapping == "prefix2" else dict(mapping=mapping)
    res = R().det(a, mode="exact", options=opts)
    assert res["exact"] == exact


def test_full_int8_12x40_exact():
    a = W.int8_12x40()
    exact = orc.radic_det_pfaffian(a.astype(np.int64))
    res = R().det(a, mode="exact")
    assert res["minors"] == math.comb(40, 12)
    assert res["n_primes"] == 3
    assert res["exact"] == exact


def test_plan_info_reports_the_default_mapping_and_depth():
    info = R().radic_plan_info(8, 32, "mixed")
    assert info["mapping"] == "prefix" and info["prefix_depth"] == 3  # m >= 7, n - m = 24 <= 3.5m
    assert R().radic_plan_info(8, 32, "fp64")["prefix_depth"] == 3
    assert R().radic_plan_info(8, 32, "pair")["prefix_depth"] == 3
    assert R().radic_plan_info(7, 40, "pair")["prefix_depth"] == 2   # n - m = 33 > 3.5m
    assert R().radic_plan_info(6, 24, "mixed")["prefix_depth"] == 2  # m < 7
    assert R().radic_plan_info(5, 60, "mixed")["prefix_depth"] == 2
    g = R().radic_plan_info(14, 20, "fp64")
    assert g["mapping"] == "group" and g["group_width"] == 16 and g["prefix_depth"] == 0
    e = R().radic_plan_info(6, 20, "exact")
    assert e["mapping"] == "prefix" and e["prefix_depth"] == 2
    t = R().radic_plan_info(6, 20, "exact", dict(mapping="thread"))
    assert t["mapping"] == "thread" and t["threads"] == 128 and t["blocks"] >= 1
    assert t["workspace_bytes"] == R().radic_workspace_bytes(6, 20, "exact", dict(mapping="thread"))


@pytest.mark.parametrize("mode", ["fp64", "mixed", "pair"])
def test_det_extreme_row_scales(mode):
    # rows far outside binary32 range, one of them subnormal in binary64: the
    # power-of-two row scaling of the staging step must keep every path exact
    # up to its rounding
    a = W.uniform_matrix(31, 5, 11)
    a[0] *= 1e-310          # subnormal binary64 entries
    a[1] *= 1e300
    a[2] *= 2.0 ** -600
    a[3, 4] = 0.0
    val, abs_sum = _exact(a)
    res = R().det(a, mode=mode, options=dict(mapping=3))
    # relative to sum|terms| (the Hadamard bound overflows binary64 here)
    tol = {"fp64": 1e-12, "mixed": 1e-5, "pair": 1e-11}[mode]
    assert abs(float(Fraction(res["value"]) - val)) <= tol * float(abs_sum)
    assert abs(res["abs_sum"] - float(abs_sum)) <= 1e-5 * float(abs_sum)
    assert_bounded(res, val)
    assert res["status"] == 0


@pytest.mark.parametrize("mode", ["mixed", "fp64", "exact"])
def test_graph_replay_equals_direct_call(mode):
    a = W.integer_matrix(41, 7, 18, 3, np.int8) if mode == "exact" else W.uniform_matrix(41, 7, 18)
    t = dev(a)
    direct = R().parse_result(R().radic_det(t, mode=mode))
    g = R().DetGraph(t, mode=mode)
    g.launch()
    g.launch()
    torch.cuda.synchronize()
    replay = R().parse_result(g.out)
    g.close()
    assert replay["value"] == direct["value"] and replay["status"] == 0
    if mode == "exact":
        assert replay["exact"] == direct["exact"]
