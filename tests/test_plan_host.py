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


# ---------------------------------------------------------------------------
# Batched path: routing and the split of every matrix's ranks into tasks
# ---------------------------------------------------------------------------


def _check_batch_tasks(tasks, shapes):
    from collections import defaultdict

    by_b = defaultdict(list)
    for t in tasks:
        by_b[t["b"]].append(t)
    for b, (m, n) in enumerate(shapes):
        ts = by_b.get(b, [])
        if m > n:
            assert not ts  # det_R = 0 with no minors
            continue
        kinds = {(t["tier"], t["kind"], t["shared"]) for t in ts}
        assert len(kinds) == 1, (b, kinds)
        _, kind, shared = kinds.pop()
        groups = defaultdict(list)
        for t in ts:
            # head-shared tasks: one task list per (last head column, segment)
            groups[(t["group"], t["vlo"], t["vhi"])].append(t)
        total = 0
        for (g, vlo, vhi), gl in groups.items():
            lim = gl[0]["lim"]
            assert all(t["lim"] == lim for t in gl)
            # 32 lanes per task, lane l takes [r0 + l*run, r0 + (l+1)*run) clipped at lim:
            # the tasks of a group tile [0, lim) without gaps or overlaps
            pos = 0
            for lo, hi in sorted((t["r0"], min(t["r0"] + 32 * t["run"], lim)) for t in gl):
                assert lo == pos and hi > lo, (b, g)
                pos = hi
            assert pos == lim
            if kind == 0:
                assert lim == math.comb(n, m)
                total += lim
            elif shared:
                # units are heads (first m-D-1 prefix columns, g the last of
                # them); a task covers the last columns v in [vlo, vhi]
                H = m - kind - 1
                assert lim == math.comb(g, H - 1)
                assert g < vlo <= vhi <= n - kind - 1
                seg = sum(math.comb(n - 1 - v, kind) for v in range(vlo, vhi + 1))
                # one lane's unit is bounded (a single prefix is never split)
                assert 0 < seg <= max(4096, math.comb(n - m + kind, kind)), (m, n, g, vlo, vhi, seg)
                total += lim * seg
            else:
                P = m - kind
                assert lim == math.comb(g, P - 1)
                total += lim * math.comb(n - 1 - g, kind)
        assert total == math.comb(n, m), (b, m, n)


def _expected_tier(m, n, tol):
    # the router's first-tier rule: binary32 when its bound envelope 1e-4
    # meets tol, pairs (m >= 3) when 2e-11 does, binary64 otherwise (the
    # device then checks each matrix's own bound)
    if 1e-4 <= tol:
        return 1
    if m >= 3 and 2e-11 <= tol:
        return 3
    return 0


@pytest.mark.parametrize("tol", [1e-10, 1e-8, 1e-4])
def test_batch_tasks_cover_every_minor_once(tol):
    from paper_1508_01326_gb300 import workloads as W

    shapes = [x.shape for x in W.batched_4096()[::4]] + [(4, 3), (1, 7), (2, 2), (10, 30), (9, 29)]
    tasks = R.batch_tasks_host(shapes, mode="mixed", tuning=R.make_tuning(tol=tol))
    _check_batch_tasks(tasks, shapes)
    tiers = {t["b"]: t["tier"] for t in tasks}
    for b, (m, n) in enumerate(shapes):
        if m <= n:
            assert tiers[b] == _expected_tier(m, n, tol), (m, n)
    # low-tier tasks come first (binary32 then pairs for each m), binary64 after
    split = [t["tier"] for t in tasks]
    first64 = split.index(0) if 0 in split else len(split)
    assert all(x != 0 for x in split[:first64]) and all(x == 0 for x in split[first64:])


def test_batch_tasks_binary64_mode_and_options():
    shapes = [(m, n) for m in range(1, 11) for n in range(m, m + 14, 3)]
    plain = R.batch_tasks_host(shapes, mode="fp64")
    _check_batch_tasks(plain, shapes)
    assert {t["tier"] for t in plain} == {0}
    # head sharing on (m - D - 1 >= 5) and off
    on = R.batch_tasks_host(shapes, mode="fp64", tuning=R.make_tuning())
    off = R.batch_tasks_host(shapes, mode="fp64", tuning=R.make_tuning(head_sharing=False))
    assert any(t["shared"] for t in on) and not any(t["shared"] for t in off)
    _check_batch_tasks(on, shapes)
    _check_batch_tasks(off, shapes)
    # per-m depth and per-minor overrides
    forced = R.batch_tasks_host(shapes, mode="mixed",
                                tuning=R.make_tuning(prefix_depth={6: 2, 9: 3}, kind={4: "thread"}, tol=1e-4))
    _check_batch_tasks(forced, shapes)
    for t in forced:
        m = shapes[t["b"]][0]
        if m == 6:
            assert t["kind"] == 2
        if m == 9:
            assert t["kind"] == 3
        if m == 4 and t["tier"] == 1:
            assert t["kind"] == 0
