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
    assert bench.prefix_ops(m, n, D) == want
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
    want = {
        "fma": heads * per_head_fma + w["prefixes"] * ((D + 1) * H + D * H) + w["cols"] * D * P
        + (3 * w["pairs"] if D == 3 else 0) + w["leaves"] * (D - 1),
        "mul": heads * per_head_mul + w["prefixes"] * (D + 1) + w["cols"] + (3 * w["pairs"] if D == 3 else 0)
        + w["leaves"],
        "add": 2 * w["leaves"],
    }
    assert bench.prefix_ops(m, n, D, shared=True) == want


def test_headline_flop_count():
    # the roofline numerator of the 8 x 32 headline (depth 3), as the bench reports it
    assert bench.prefix_flops(8, 32, 3) == 154415430
    assert bench.prefix_ops(8, 32, 3)["add"] == 2 * math.comb(32, 8)
