"""GPU parity of the batched path: every matrix of a batch against the oracle.

Small batches of uneven shapes are checked against the exact enumeration of
Eq. (1); the full 4096-matrix workload is checked against the exact values
of tests/golden/workload_exact.txt (written by the oracle's Pfaffian closed
form).  Binary64 results must be within 1e-12 * sum|terms|; mixed results
within 1e-10 * sum|terms| (the target the tier router is built for); results
of the pair tier (elimination in pairs of binary32) within 1e-11 * sum|terms|.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle.radic_oracle as orc
from paper_1508_01326_gb300 import workloads as W
from tests.conftest import ROOT, golden_abs_sums

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1508_01326_gb300 import build as B

    B.build()


def R():
    import paper_1508_01326_gb300 as R_

    return R_


def small_batch(seed, count, max_m=10, max_d=6):
    rng = np.random.default_rng(seed)
    mats = []
    for _ in range(count):
        m = int(rng.integers(1, max_m + 1))
        n = int(m + rng.integers(-1, max_d + 1))
        n = max(n, 1)
        mats.append(rng.standard_normal((m, n)))
    return mats


def assert_bounded(r, exact):
    """The result's err_bound is an upper bound on its actual error against the exact value."""
    err = abs(Fraction(r["value"]) - Fraction(exact))
    assert err <= Fraction(r["err_bound"]), (float(err), r["err_bound"])


def run_batch(mats, mode, dtype=np.float64, tuning=None, graph=False):
    data, ms, ns, offs = W.pack_batch(mats, dtype)
    A = torch.from_numpy(data).cuda()
    plan = R().BatchPlan(list(zip(ms, ns)), offs, mode=mode, tuning=tuning)
    if graph:
        out = plan.new_results()
        g = plan.graph(A, out)
        g.launch()
        g.launch()
    else:
        out = plan.radic_det_batched(A)
    torch.cuda.synchronize()
    res = R().parse_results(out)
    info = plan.info()
    plan.close()
    return res, info


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_small_batch_matches_oracle(mode):
    mats = small_batch(1, 60)
    res, info = run_batch(mats, mode)
    for a, r in zip(mats, res):
        val, abs_sum = orc.radic_det_exact(a)
        m, n = a.shape
        assert r["minors"] == (math.comb(n, m) if m <= n else 0)
        assert r["status"] == 0
        if m > n:
            assert r["value"] == 0.0
            continue
        if r["tier"] == 0:  # binary64
            assert abs(Fraction(r["value"]) - val) <= Fraction(1e-12) * abs_sum
        elif r["tier"] == 3:  # pairs of binary32
            assert abs(float(Fraction(r["value"]) - val)) <= 1e-11 * float(abs_sum)
        else:
            # small matrices are routed to binary64 by the mixed plan
            assert abs(float(Fraction(r["value"]) - val)) <= 1e-10 * float(abs_sum)
        assert_bounded(r, val)
        if mode == "mixed":  # the device check keeps every bound within the plan's target
            assert r["err_bound"] <= 1e-10 * float(abs_sum) * (1 + 1e-9)
    if mode == "fp64":
        assert info["matrices_fp32"] == 0


def test_small_batch_graph_equals_direct_call():
    mats = small_batch(2, 40)
    direct, _ = run_batch(mats, "fp64")
    graphed, _ = run_batch(mats, "fp64", graph=True)
    assert [r["value"] for r in direct] == [r["value"] for r in graphed]


def test_batch_with_per_minor_tuning_and_float32_input():
    mats = [W.uniform_matrix(s, m, n) for s, (m, n) in enumerate([(3, 9), (5, 11), (8, 13), (2, 12), (1, 7)])]
    tuning = R().make_tuning(kind={m: "thread" for m in range(1, 9)}, task_cost={m: 2000 for m in range(1, 11)},
                             tol=1.0)  # tol 1: every matrix in the binary32 tier
    res, info = run_batch(mats, "mixed", dtype=np.float32, tuning=tuning)
    assert info["matrices_fp32"] == len(mats)
    for a, r in zip(mats, res):
        a32 = a.astype(np.float32)
        val, abs_sum = orc.radic_det_exact(a32)
        assert r["tier"] == 1
        m = a.shape[0]
        assert abs(float(Fraction(r["value"]) - val)) <= 8 * m * 2.0 ** -24 * float(abs_sum) * 4
        assert_bounded(r, val)


@pytest.mark.parametrize("depth", [2, 3])
def test_batch_prefix_depths_match_oracle(depth):
    mats = small_batch(4, 40, max_m=10, max_d=8)
    tuning = R().make_tuning(prefix_depth={m: depth for m in range(3, 11)}, task_cost={m: 3000 for m in range(1, 11)})
    res, _ = run_batch(mats, "fp64", tuning=tuning)
    for a, r in zip(mats, res):
        val, abs_sum = orc.radic_det_exact(a)
        assert abs(Fraction(r["value"]) - val) <= Fraction(1e-12) * abs_sum
        assert_bounded(r, val)


@pytest.mark.parametrize("mode,tiers", [("fp64", None), ("mixed", ["pair"]), ("mixed", ["fp32"])])
@pytest.mark.parametrize("head_sharing", [True, False])
def test_batch_head_sharing_matches_oracle(mode, tiers, head_sharing):
    mats = small_batch(8, 40, max_m=10, max_d=10)
    kw = dict(head_sharing=head_sharing, task_cost={m: 5000 for m in range(1, 11)})
    if mode == "mixed":
        kw.update(tiers=tiers, tol=1.0 if tiers == ["fp32"] else 1e-10)
    res, _ = run_batch(mats, mode, tuning=R().make_tuning(**kw))
    for a, r in zip(mats, res):
        val, abs_sum = orc.radic_det_exact(a)
        m = a.shape[0]
        tol = {0: 1e-12, 3: 1e-11}.get(r["tier"], 8 * m * 2.0 ** -24)
        assert abs(float(Fraction(r["value"]) - val)) <= tol * float(abs_sum)
        assert_bounded(r, val)


def test_batch_is_deterministic():
    mats = small_batch(3, 50, max_d=12)
    tuning = R().make_tuning(tol=1.0)
    a, _ = run_batch(mats, "mixed", tuning=tuning)
    b, _ = run_batch(mats, "mixed", tuning=tuning)
    assert [r["value"] for r in a] == [r["value"] for r in b]


def test_batch_flagged_task_recomputed_in_binary64():
    # Wilkinson's growth matrix in the leading 9 columns of a 9 x 16 matrix:
    # the prefixes through those columns flag and their tasks are redone in
    # binary64 by the second kernel.
    m = 9
    w = np.eye(m) - np.tril(np.ones((m, m)), -1)
    w[:, -1] = 1.0
    a = np.concatenate([w, W.uniform_matrix(77, m, 7)], axis=1)
    tuning = R().make_tuning(tol=1.0)
    res, info = run_batch([a, W.uniform_matrix(78, 4, 10)], "mixed", tuning=tuning)
    val, abs_sum = orc.radic_det_exact(a)
    assert res[0]["flagged"] > 0
    assert abs(float(Fraction(res[0]["value"]) - val)) <= 8 * m * 2.0 ** -24 * float(abs_sum)


def test_batch_flagged_pair_task_recomputed_in_binary64():
    m = 9
    w = np.eye(m) - np.tril(np.ones((m, m)), -1)
    w[:, -1] = 1.0
    a = np.concatenate([w, W.uniform_matrix(79, m, 7)], axis=1)
    tuning = R().make_tuning(tiers=["pair"], tol=1e-10)
    res, info = run_batch([a, W.uniform_matrix(80, 5, 12)], "mixed", tuning=tuning)
    assert info["matrices_pair"] == 2
    val, abs_sum = orc.radic_det_exact(a)
    assert res[0]["flagged"] > 0
    assert abs(float(Fraction(res[0]["value"]) - val)) <= 1e-12 * float(abs_sum)


def test_batch_flagged_per_minor_task_recomputed_in_binary64():
    # per-minor binary32 tasks (m = 8) through the growth matrix: the flagged
    # tasks are redone by the binary64 kernel with the per-minor mapping.  The
    # rows are scaled to a largest entry of 1/2, so the last pivot of the
    # growth minor is 2^7 / 2 = 64: a threshold of 16 flags it.
    m = 8
    w = np.eye(m) - np.tril(np.ones((m, m)), -1)
    w[:, -1] = 1.0
    a = np.concatenate([w, W.uniform_matrix(81, m, 4)], axis=1)
    tuning = R().make_tuning(kind={8: "thread"}, task_cost={8: 2000}, tol=1.0, growth_threshold=16.0)
    res, info = run_batch([a], "mixed", tuning=tuning)
    assert info["matrices_fp32"] == 1
    val, abs_sum = orc.radic_det_exact(a)
    assert res[0]["flagged"] > 0
    assert abs(float(Fraction(res[0]["value"]) - val)) <= 8 * m * 2.0 ** -24 * float(abs_sum)


def _golden(name):
    vals = {}
    with open(os.path.join(ROOT, "tests", "golden", "workload_exact.txt")) as f:
        for line in f:
            p = line.split()
            if p and p[0] == name:
                vals[int(p[1])] = float(p[4])
    return [vals[i] for i in range(len(vals))]


@pytest.mark.parametrize("mode,dtype,golden,tol", [
    ("mixed", np.float32, "batched_4096_f32", 1e-10),
    ("mixed", np.float64, "batched_4096_f64", 1e-10),
    ("mixed", np.float32, "batched_4096_f32", 1e-4),
    ("fp64", np.float64, "batched_4096_f64", 1e-12),
])
def test_full_batched_4096(mode, dtype, golden, tol):
    mats = W.batched_4096()
    want = _golden(golden)
    # tolerance scale: the oracle's sum|terms| of each matrix (binary64 host
    # enumeration, tests/golden/workload_abs_sum.txt), not the GPU's own sum
    scale = golden_abs_sums(golden)
    tuning = R().make_tuning(tol=tol) if mode == "mixed" else None
    res, info = run_batch(mats, mode, dtype=dtype, tuning=tuning)
    worst = 0.0
    for r, w, s in zip(res, want, scale):
        assert r["status"] == 0
        if s == 0.0:
            assert r["value"] == 0.0 and r["abs_sum"] == 0.0
            continue
        worst = max(worst, abs(r["value"] - w) / s)
        # the a-posteriori bound holds (against the correctly rounded exact
        # value, so up to half an ulp of it); in the mixed mode it meets the
        # target (the device check redoes in binary64 what does not), and
        # binary64 bounds stay below 1e-10 (the errors themselves are checked
        # against 1e-12 below)
        assert abs(r["value"] - w) <= r["err_bound"] + 0.5 * math.ulp(w), (r, w)
        assert r["err_bound"] <= (tol if mode == "mixed" else 1e-10) * s * (1 + 1e-5), (r, s)
        # the GPU's magnitude sum agrees with the oracle's: binary64 to 1e-9;
        # binary32 elimination to 1e-5 (each |term| carries its minor's
        # rounding); pairs to 1e-6 (their magnitudes are summed in binary32)
        assert abs(r["abs_sum"] - s) <= {1: 1e-5, 3: 1e-6}.get(r["tier"], 1e-9) * s, (r, s)
    assert worst <= tol, worst
    assert info["matrices_fp32"] + info["matrices_pair"] + info["matrices_fp64"] == len(mats)
    if mode == "mixed":
        # first tier: binary32 when 1e-4 meets tol, else pairs (m >= 3) when
        # 2e-11 does, else binary64; the device check then redoes in binary64
        # every matrix whose bound misses tol
        want32 = want_pair = 0
        for a in mats:
            m, n = a.shape
            if m > n:
                continue
            if 1e-4 <= tol:
                want32 += 1
            elif m >= 3 and 2e-11 <= tol:
                want_pair += 1
        assert info["matrices_fp32"] == want32
        assert info["matrices_pair"] == want_pair
        if tol >= 1e-4:
            assert want32 > 0
        if tol <= 1e-10:
            assert want_pair > 0
    else:
        assert info["matrices_pair"] == 0


def test_pair_tier_small_batch_matches_oracle():
    mats = small_batch(5, 60, max_m=10, max_d=10)
    tuning = R().make_tuning(tiers=["pair"], tol=1e-10)
    res, info = run_batch(mats, "mixed", tuning=tuning)
    assert info["matrices_fp32"] == 0
    assert info["matrices_pair"] == sum(1 for a in mats if 3 <= a.shape[0] <= a.shape[1])
    for a, r in zip(mats, res):
        val, abs_sum = orc.radic_det_exact(a)
        m, n = a.shape
        assert r["status"] == 0
        if m > n:
            assert r["value"] == 0.0
            continue
        # pairs for m >= 3, unless the device check redid the matrix in binary64
        assert r["tier"] in ((3, 0) if m >= 3 else (0,))
        assert abs(float(Fraction(r["value"]) - val)) <= 1e-11 * float(abs_sum)
        assert_bounded(r, val)
        assert r["err_bound"] <= 1e-10 * float(abs_sum) * (1 + 1e-9)


@pytest.mark.parametrize("depth", [2, 3])
def test_pair_tier_both_depths(depth):
    mats = small_batch(6, 30, max_m=10, max_d=8)
    mats = [a for a in mats if a.shape[0] >= 4]
    tuning = R().make_tuning(tiers=["pair"], tol=1e-10, prefix_depth={m: depth for m in range(4, 11)},
                             task_cost={m: 3000 for m in range(1, 11)})
    res, info = run_batch(mats, "mixed", tuning=tuning)
    for a, r in zip(mats, res):
        val, abs_sum = orc.radic_det_exact(a)
        if a.shape[0] > a.shape[1]:
            continue
        assert r["tier"] in (3, 0)  # pairs, or binary64 after the device check
        assert abs(float(Fraction(r["value"]) - val)) <= 1e-11 * float(abs_sum)
        assert_bounded(r, val)


def test_fp32_only_router_sends_the_rest_to_binary64():
    mats = small_batch(7, 30)
    res, info = run_batch(mats, "mixed", tuning=R().make_tuning(tiers=["fp32"], tol=1e-10))
    assert info["matrices_pair"] == 0
    assert all(r["tier"] in (0, 1) for r in res)


def structured_batch(seed):
    """Inputs on which per-minor rounding errors do not behave like independent
    random variables: nearly repeated columns, columns equal up to their last
    bits, low rank plus a small perturbation, and column pairs whose terms
    cancel across the whole sum."""
    rng = np.random.default_rng(seed)
    mats = []
    for m, n in [(4, 11), (5, 12), (6, 12), (7, 13), (8, 14), (6, 14)]:
        a = rng.standard_normal((m, n))
        a[:, 1::3] = a[:, 0:-1:3][:, : a[:, 1::3].shape[1]] + 1e-9 * rng.standard_normal((m, a[:, 1::3].shape[1]))
        mats.append(a)
        b = rng.standard_normal((m, n))
        b[:, 1::2] = b[:, 0:-1:2][:, : b[:, 1::2].shape[1]] * (1.0 + 2.0 ** -40)
        mats.append(b)
        r = m - 2
        c = rng.standard_normal((m, r)) @ rng.standard_normal((r, n)) + 1e-4 * rng.standard_normal((m, n))
        mats.append(c)
        half = n // 2
        d0, d1 = rng.uniform(-1, 1, (m, half)), rng.uniform(-1, 1, (m, half))
        d = np.empty((m, 2 * half))
        d[:, 0::2], d[:, 1::2] = d0, d0 + 0.25 * d1
        mats.append(d)
    return mats


def test_structured_inputs_bound_holds_and_rerouting_keeps_target():
    # The first tier of every matrix here is pairs of binary32 (tol 1e-10);
    # the device check sends a matrix to binary64 when its own bound misses
    # the target.  Every result's bound must hold, and every result must meet
    # the target, or be a binary64 result whose own bound says why not.
    mats = structured_batch(11)
    tol = 1e-10
    res, info = run_batch(mats, "mixed", tuning=R().make_tuning(tol=tol))
    assert info["matrices_pair"] == len(mats)
    rerouted = 0
    for a, r in zip(mats, res):
        val, abs_sum = orc.radic_det_exact(a)
        assert r["status"] == 0
        assert_bounded(r, val)
        err = abs(float(Fraction(r["value"]) - val))
        if r["err_bound"] <= tol * float(abs_sum) * (1 + 1e-9):
            assert err <= tol * float(abs_sum)
        else:
            assert r["tier"] == 0, r
        rerouted += r["tier"] == 0
    assert rerouted >= 1
