"""Host logic of the batched autotuner without a GPU: candidate sets, the choice
of the fastest candidate per m, and the on-disk cache (timings are faked)."""
import numpy as np
import pytest

from paper_1508_01326_gb300 import autotune as AT


def test_candidates_per_m():
    costs = (1000.0, 2000.0)
    # m <= 2: per-minor only; m = 3: depth-2 prefixes (and per-minor in the
    # binary32 tier); m >= 4: depths 2 and 3; per-minor only up to m = 8
    assert {k for k, _, _ in AT.candidates(2, False, costs)} == {"thread"}
    assert {(k, d) for k, d, _ in AT.candidates(3, True, costs)} == {("prefix", 2), ("thread", 0)}
    assert {(k, d) for k, d, _ in AT.candidates(3, False, costs)} == {("prefix", 2)}
    assert {(k, d) for k, d, _ in AT.candidates(8, True, costs)} == {("prefix", 2), ("prefix", 3), ("thread", 0)}
    assert {(k, d) for k, d, _ in AT.candidates(9, True, costs)} == {("prefix", 2), ("prefix", 3)}
    assert len(AT.candidates(6, False, costs)) == 2 * 2  # two kinds x two costs


def test_autotune_picks_fastest_and_caches(monkeypatch, tmp_path):
    timed = []

    def fake_time(mats, mode, dtype, tuning, reps=3):
        m = int(mats[0].shape[0])
        kind = int(tuning.kind[m])
        depth = int(tuning.prefix_depth[m])
        cost = float(tuning.task_cost[m])
        timed.append((m, kind, depth, cost))
        # depth 3 with task cost 12000 is fastest for m = 6; per-minor for m = 2
        return 1.0 + (0.0 if (depth == 3 and cost == 12000.0) else 0.5) + 0.001 * m

    monkeypatch.setattr(AT, "_time_plan", fake_time)
    monkeypatch.setattr(AT.torch.cuda, "get_device_name", lambda *a, **k: "fake-gpu")
    rng = np.random.default_rng(0)
    mats = [rng.uniform(-1, 1, (6, 14)), rng.uniform(-1, 1, (6, 12)), rng.uniform(-1, 1, (2, 9))]
    path = str(tmp_path / "tune.json")
    tun, table = AT.autotune(mats, mode="mixed", tol=1e-10, path=path)
    assert table["6"]["kind"] == "prefix" and table["6"]["depth"] == 3 and table["6"]["task_cost"] == 12000.0
    assert table["2"]["kind"] == "thread"
    assert int(tun.prefix_depth[6]) == 3 and float(tun.task_cost[6]) == 12000.0
    n_timed = len(timed)
    assert n_timed == len(AT.candidates(6, False, AT.DEFAULT_COSTS)) + len(AT.candidates(2, False, AT.DEFAULT_COSTS))
    # the second call reads the cache and times nothing
    tun2, table2 = AT.autotune(mats, mode="mixed", tol=1e-10, path=path)
    assert len(timed) == n_timed and table2 == table
    # another tolerance is another cache entry
    AT.autotune(mats[:1], mode="mixed", tol=1e-6, path=path)
    assert len(timed) > n_timed
