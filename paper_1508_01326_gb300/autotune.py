"""Autotuner of the batched path: per m, the minor-to-warp mapping, prefix depth and task size.

For every m present in a batch it times the batched call on the sub-batch of
matrices with that m under each candidate (mapping, prefix depth, task cost)
and keeps the fastest.  Results are cached in a JSON file keyed by GPU name, mode, target
tolerance and input dtype (default ~/.cache/radic_gb300/autotune.json, or the
path in RADIC_AUTOTUNE_CACHE).  Host logic only; timing uses CUDA events
around the library's own launches.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Iterable, List, Optional, Tuple

import numpy as np
import torch

from . import api
from . import workloads as W

DEFAULT_COSTS = (4000.0, 12000.0, 30000.0, 80000.0)


def cache_path() -> str:
    return os.environ.get("RADIC_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "radic_gb300", "autotune.json"))


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, data: dict) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_plan(mats: List[np.ndarray], mode: str, dtype, tuning, reps: int = 3) -> float:
    data, ms, ns, offs = W.pack_batch(mats, dtype)
    A = torch.from_numpy(data).cuda()
    plan = api.BatchPlan(list(zip(ms, ns)), offs, mode=mode, tuning=tuning)
    out = plan.new_results()
    plan.radic_det_batched(A, out)  # warm-up
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.radic_det_batched(A, out)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    plan.close()
    return best


def candidates(m: int, tier_fp32: bool, costs: Iterable[float]) -> List[Tuple[str, int, float]]:
    """(mapping, prefix depth (0 for the per-minor mapping), task cost) triples to time for this m."""
    kinds = []
    if m >= 3:
        kinds.append(("prefix", 2))
    if m >= 4:
        kinds.append(("prefix", 3))
    if m <= 2 or (tier_fp32 and m <= 8):
        kinds.append(("thread", 0))
    return [(k, d, c) for k, d in kinds for c in costs]


def autotune(mats: List[np.ndarray], mode: str = "mixed", tol: float = 1e-10, dtype=np.float64,
             costs: Iterable[float] = DEFAULT_COSTS, path: Optional[str] = None, force: bool = False,
             reps: int = 3) -> Tuple["api.L.RadicBatchTuning", dict]:
    """Returns (tuning struct, table {m: {"kind", "depth", "task_cost", "ms"}}) for this batch."""
    path = path or cache_path()
    dev = torch.cuda.get_device_name()
    key = f"{dev}|{mode}|{tol:g}|{np.dtype(dtype).name}|v3"
    cache = _load(path)
    table: Dict[str, dict] = dict(cache.get(key, {}))
    by_m: Dict[int, List[np.ndarray]] = {}
    for a in mats:
        by_m.setdefault(int(a.shape[0]), []).append(a)
    changed = False
    for m, group in sorted(by_m.items()):
        if str(m) in table and not force:
            continue
        # is any matrix of this m routed to the binary32 tier?  (the plan's
        # first-tier rule: binary32 when its bound envelope 1e-4 meets tol)
        tier_fp32 = mode == "mixed" and tol >= 1e-4 and any(a.shape[0] <= a.shape[1] for a in group)
        best = None
        for kind, depth, cost in candidates(m, tier_fp32, costs):
            tun = api.make_tuning(kind={m: kind}, task_cost={m: cost}, prefix_depth={m: depth}, tol=tol)
            ms = _time_plan(group, mode, dtype, tun, reps)
            if best is None or ms < best["ms"]:
                best = {"kind": kind, "depth": depth, "task_cost": cost, "ms": ms}
        table[str(m)] = best
        changed = True
    if changed:
        cache[key] = table
        _store(path, cache)
    tun = api.make_tuning(kind={int(m): v["kind"] for m, v in table.items()},
                          task_cost={int(m): v["task_cost"] for m, v in table.items()},
                          prefix_depth={int(m): v.get("depth", 0) for m, v in table.items()}, tol=tol)
    return tun, table
