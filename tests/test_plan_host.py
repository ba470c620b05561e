"""Host-only checks of the prefix mapping's task table (no GPU).

The prefix kernels split the C(n,m) minors of Eq. (1) into contiguous runs
(Section 5), here runs of prefixes: a prefix is the first m-D columns of a
sequence, grouped by its last column v, and its leaves are the C(n-1-v, D)
choices of the D later columns.  radic_prefix_plan_host plans that table for
a given SM count and residency without touching a GPU; these tests check
that every minor belongs to exactly one planned prefix and that every prefix
of a group falls in exactly one task, at the full sizes the bench uses.
"""
import math

import pytest

import paper_1508_01326_gb300 as R

SHAPES = [
    (8, 32, "mixed"), (8, 32, "pair"), (8, 32, "fp64"), (7, 30, "mixed"), (9, 28, "mixed"), (10, 30, "mixed"),
    (12, 28, "mixed"), (6, 40, "mixed"), (10, 24, "exact"), (12, 40, "exact"), (3, 12, "fp64"), (5, 60, "mixed"),
]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1508_01326_gb300 import build as B

    B.build()


@pytest.mark.parametrize("m,n,mode", SHAPES)
@pytest.mark.parametrize("per_sm", [1, 3, 4])
def test_prefix_groups_cover_every_minor_once(m, n, mode, per_sm):
    plan = R.prefix_plan_host(m, n, mode, sms=152, blocks_per_sm=per_sm)
    D = plan["depth"]
    P = m - D
    assert D in (2, 3) and P >= 1
    # groups: v = P-1 .. n-1-D, each with C(v, P-1) prefixes of C(n-1-v, D) leaves
    assert (plan["v_lo"], plan["v_hi"]) == (P - 1, n - 1 - D)
    total = 0
    for v, g in plan["groups"].items():
        assert g["count"] == math.comb(v, P - 1)
        total += g["count"] * math.comb(n - 1 - v, D)
    assert total == math.comb(n, m)


@pytest.mark.parametrize("m,n,mode", SHAPES)
@pytest.mark.parametrize("per_sm", [1, 3, 4])
def test_prefix_tasks_cover_every_prefix_once(m, n, mode, per_sm):
    plan = R.prefix_plan_host(m, n, mode, sms=152, blocks_per_sm=per_sm)
    vs = sorted(plan["groups"])
    starts = [plan["groups"][v]["task_start"] for v in vs] + [plan["tasks"]]
    assert starts[0] == 0
    for i, v in enumerate(vs):
        g = plan["groups"][v]
        lp, run = g["lanes"], g["run"]
        assert lp in (1, 2, 4, 8, 16, 32) and run >= 1
        if plan["depth"] == 2:
            assert lp == 1  # depth-2 prefixes are not split
        tasks = starts[i + 1] - starts[i]
        per_task = (32 // lp) * run  # lane groups of a warp x prefixes per group
        # the group's prefixes fill its tasks in order, and no task is empty
        assert tasks * per_task >= g["count"]
        assert (tasks - 1) * per_task < g["count"]
    assert 1 <= plan["blocks"] <= 152 * per_sm


def test_prefix_plan_options():
    base = R.prefix_plan_host(8, 32, "mixed")
    assert base["dynamic"]
    det = R.prefix_plan_host(8, 32, "mixed", options=dict(deterministic=True))
    assert not det["dynamic"]
    assert det["groups"] == base["groups"] and det["tasks"] == base["tasks"]
    forced = R.prefix_plan_host(8, 32, "mixed", options=dict(lanes_per_prefix=8))
    assert all(g["lanes"] == 8 for g in forced["groups"].values())
    assert R.prefix_plan_host(8, 32, "mixed", options=dict(prefix_depth=2))["depth"] == 2
    # heavy groups (the most candidate columns) get more lanes than light ones
    groups = base["groups"]
    assert groups[base["v_lo"]]["lanes"] >= groups[base["v_hi"]]["lanes"]
    # depth 3 needs a prefix of at least one column
    with pytest.raises(R.RadicError):
        R.prefix_plan_host(3, 10, "mixed", options=dict(prefix_depth=3))
