"""The bench's algorithmic operation counts (the roofline numerator) against an
explicit walk over the prefixes and leaves they aggregate (no GPU)."""
import itertools
import math

import pytest

import bench


def _walk(m, n, D, shared=False):
    """Counts of prefixes (or heads and extensions), candidate columns, column
    pairs and leaves, by enumerating every column sequence of Eq. (1)."""
    P = m - D
    prefixes = set()
    heads = set()
    leaves = 0
    for J in itertools.combinations(range(n), m):
        prefixes.add(J[:P])
        heads.add(J[:P - 1])
        leaves += 1
    cols = pairs = 0
    for pre in prefixes:
        k = n - 1 - pre[-1]
        cols += k
        pairs += math.comb(k, 2)
    return {"prefixes": len(prefixes), "heads": len(heads), "cols": cols, "pairs": pairs, "leaves": leaves}


@pytest.mark.parametrize("m,n,D", [(3, 8, 2), (4, 9, 2), (4, 9, 3), (5, 11, 3), (6, 10, 3), (8, 12, 3)])
def test_prefix_ops_aggregate_every_prefix_and_leaf(m, n, D):
    w = _walk(m, n, D)
    assert w["leaves"] == math.comb(n, m)
    P = m - D
    per_prefix_fma = sum((m - k - 1) * (P - k - 1) for k in range(P)) + D * P * (P - 1) // 2
    per_prefix_mul = sum(m - k - 1 for k in range(P)) + P
    want = {
        "fma": w["prefixes"] * per_prefix_fma + w["cols"] * D * P + (3 * w["pairs"] if D == 3 else 0)
        + w["leaves"] * (D - 1),
        "mul": w["prefixes"] * per_prefix_mul + w["cols"] + (3 * w["pairs"] if D == 3 else 0) + w["leaves"],
        "add": 2 * w["leaves"],
    }
    got = bench.prefix_ops(m, n, D)
    assert (got["all_fma"], got["all_mul"], got["all_add"]) == (want["fma"], want["mul"], want["add"])
    # the prefix factorisations alone
    assert (got["pre_fma"], got["pre_mul"]) == (w["prefixes"] * per_prefix_fma, w["prefixes"] * per_prefix_mul)
    assert bench.prefix_flops(m, n, D) == 2 * want["fma"] + want["mul"] + want["add"]


@pytest.mark.parametrize("m,n,D", [(8, 13, 2), (9, 14, 3), (10, 14, 3)])
def test_prefix_ops_head_sharing_aggregate(m, n, D):
    # with head sharing every head (first m-D-1 columns) is factored once and
    # every prefix is one extension of its head; columns, pairs and leaves as
    # without sharing
    w = _walk(m, n, D)
    P, H = m - D, m - D - 1
    per_head_fma = sum((m - k - 1) * (H - k - 1) for k in range(H)) + (D + 1) * H * (H - 1) // 2
    per_head_mul = sum(m - k - 1 for k in range(H)) + H
    # heads that have at least one prefix with a leaf (last head column <= n-D-2)
    heads = sum(math.comb(u, H - 1) for u in range(H - 1, n - D - 1))
    assert heads == w["heads"]
    want = {
        "fma": heads * per_head_fma + w["prefixes"] * ((D + 1) * H + D * H) + w["cols"] * D * P
        + (3 * w["pairs"] if D == 3 else 0) + w["leaves"] * (D - 1),
        "mul": heads * per_head_mul + w["prefixes"] * (D + 1) + w["cols"] + (3 * w["pairs"] if D == 3 else 0)
        + w["leaves"],
        "add": 2 * w["leaves"],
    }
    got = bench.prefix_ops(m, n, D, shared=True)
    assert (got["all_fma"], got["all_mul"], got["all_add"]) == (want["fma"], want["mul"], want["add"])
    assert (got["pre_fma"], got["pre_mul"]) == (heads * per_head_fma + w["prefixes"] * ((D + 1) * H + D * H),
                                                heads * per_head_mul + w["prefixes"] * (D + 1))
    assert got["upd_fma"] == w["prefixes"] * D * H
    # the pair tier: columns, pairs, leaves and the extensions' W updates in
    # binary32 flops of the pair algorithms, the rest of the prefix part in
    # binary64 flops
    f = bench.pair_flops(m, n, D, shared=True)
    assert f["fp64"] == 2 * (got["pre_fma"] - got["upd_fma"]) + got["pre_mul"]
    assert f["fp32"] == 18 * (got["fma"] + got["upd_fma"]) + 10 * got["mul"] + 12 * w["leaves"]


def test_single_matrix_flop_count():
    # the prefix path's flops on the 8 x 32 workload (depth 3)
    assert bench.prefix_flops(8, 32, 3) == 154415430
    assert bench.prefix_ops(8, 32, 3)["add"] == 2 * math.comb(32, 8)


@pytest.mark.parametrize("m,n,D,K", [(5, 11, 2, 1), (6, 12, 3, 2), (10, 15, 3, 3), (12, 16, 3, 3)])
def test_modp_multiplies_aggregate_every_prefix_and_leaf(m, n, D, K):
    # 32-bit multiplies of the exact prefix path, against a walk over the prefixes
    w = _walk(m, n, D)
    P = m - D
    per_pre = 4 * sum((m - 1 - k) * (P - 1 - k) for k in range(P)) + 3 * (2 * P + D - 1) + 9
    per_col = 4 * sum(m - 1 - k for k in range(P)) + 5
    want = K * (w["prefixes"] * per_pre + w["cols"] * per_col + (12 * w["pairs"] if D == 3 else 0)
                + w["leaves"] * (7 if D == 3 else 4))
    assert bench.modp_mults(m, n, D, K) == want
