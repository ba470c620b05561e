#!/usr/bin/env python
"""Benchmark of Radic's determinant on one GB300 (or N, one process each).

One step = one radic_det_batched call over the 4096-matrix batch (m uniform
in 2..10, n = m + 1..20, binary64 entries N(0,1), 3,373,693,081 signed minors
in all) through the MIXED router at a target error bound of 1e-10 of
sum|terms|: stage each matrix and its binomial table, split its ranks into
warp tasks, unrank, step with the successor, gather, factor (prefixes in
binary64, Schur-complement columns and leaves in pairs of binary32; m <= 2
in binary64), sign, accumulate with the running error bound, check every
matrix's bound on the device and redo in binary64 the matrices that miss the
target, reduce.  The headline `value` is signed minors per second of that
step.  Beside it: the plain binary64 batched path and one plain binary64
launch per matrix on the same batch, the other configurations (8 x 32
single matrix in every mode, exact 12 x 40, exact 3 x 12 latency, forward and
backward of 256 x 6 x 28), the measured pipe peaks, the roofline of the
dominant kernel, the end-to-end call from host memory and the oracle on the
host cores.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run; every rank computes its own
batch (independent problems, weak scaling, no collective on the data path)
and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "signed minors/sec & % FMA peak, mixed vs plain FP64 GPU at stated rel err"
UNIT = "minors/s"
TOL = 1e-10
WORKLOAD = ("batched_4096: 4096 matrices, m uniform in {2..10}, n = m + uniform{1..20}, binary64 entries "
            "N(0,1) from numpy PCG64 seed 4, 3,373,693,081 signed minors; MIXED router at err_bound <= 1e-10 "
            "of sum|terms| per matrix")
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# dominant kernel (the pair tier's m = 10 group of the 4096-matrix batch)
# from one ncu capture of that kernel on the same 493 matrices
# (`cli --batched-m 10 --mode mixed`): 7.301 MB read + 0.080 MB written.  Set to None whenever that kernel changes until it is recaptured.
DOMINANT_DRAM_BYTES = 7_381_248
ORACLE_SAMPLE_OFFSET = 1_000_000


# ---------------------------------------------------------------------------
# golden values (written by tests/golden/*.py from oracle/ only)
# ---------------------------------------------------------------------------
def _golden_rows(fname: str, name: str) -> dict:
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", fname)) as f:
        for line in f:
            p = line.split()
            if p and p[0] == name:
                out[int(p[1])] = p
    return out


def golden_values(name: str) -> list:
    rows = _golden_rows("workload_exact.txt", name)
    return [float(rows[i][4]) for i in range(len(rows))]


def golden_fraction(name: str):
    from fractions import Fraction

    p = _golden_rows("workload_exact.txt", name)[0]
    return Fraction(int(p[2]), int(p[3]))


def golden_abs_sums(name: str) -> list:
    rows = _golden_rows("workload_abs_sum.txt", name)
    return [float(rows[i][2]) for i in range(len(rows))]


# ---------------------------------------------------------------------------
# clocks sampled with nvidia-smi while the GPU works
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic operation counts (roofline numerators; tests/test_bench_counts.py
# checks them against explicit walks over the minors)
# ---------------------------------------------------------------------------
def prefix_ops(m: int, n: int, D: int, shared: bool = False) -> dict:
    """Operation counts of the prefix-sharing path with depth D (2 or 3).

    Per (m-D)-column prefix: the partial-pivot elimination of its m x (m-D)
    matrix (multipliers and FMA updates), the product of pivots and
    W = -L21 L11^-1 (FMAs); per candidate column: its D Schur-complement
    entries (FMAs) and the scale (a multiply); per column pair (D = 3): a cross
    product (three multiplies, three FMAs); per leaf minor: the D x D
    determinant (D = 2: a multiply and an FMA; D = 3: a multiply and two
    FMAs) and two additions into the sums (signed and absolute).

    With `shared` (head sharing of the batched path) each head of H = m-D-1
    columns is factored once (its elimination and W1 for the D+1 rows left)
    and each last prefix column costs one elimination step: the D+1
    Schur-complement entries of the column, D multipliers and the D x H
    update of W, one multiply into the pivot product.

    Returns the counts split into the prefix part ("pre_fma", "pre_mul":
    factorisations, extensions; "upd_fma": the share of pre_fma in the
    extensions' D x H update of W, which the pair tier runs in pairs of
    binary32)
    and the rest ("fma", "mul", "add": columns, column pairs, leaves), plus
    their totals under "all_*".
    """
    P = m - D
    pre = {"fma": sum((m - k - 1) * (P - k - 1) for k in range(P)) + D * P * (P - 1) // 2,
           "mul": sum(m - k - 1 for k in range(P)) + P}
    col = {"fma": D * P, "mul": 1}
    pair = {"fma": 3, "mul": 3} if D == 3 else {"fma": 0, "mul": 0}
    leaf = {"fma": D - 1, "mul": 1, "add": 2}
    tot = {"pre_fma": 0, "pre_mul": 0, "upd_fma": 0, "fma": 0, "mul": 0, "add": 0}

    def body(cnt, k):
        tot["fma"] += cnt * (k * col["fma"] + math.comb(k, 2) * pair["fma"] + math.comb(k, D) * leaf["fma"])
        tot["mul"] += cnt * (k * col["mul"] + math.comb(k, 2) * pair["mul"] + math.comb(k, D) * leaf["mul"])
        tot["add"] += cnt * math.comb(k, D) * leaf["add"]

    if shared:
        H = P - 1
        head = {"fma": sum((m - k - 1) * (H - k - 1) for k in range(H)) + (D + 1) * H * (H - 1) // 2,
                "mul": sum(m - k - 1 for k in range(H)) + H}
        ext = {"fma": (D + 1) * H + D * H, "mul": D + 1}
        for u in range(H - 1, n - D - 1):
            cnt = math.comb(u, H - 1)
            tot["pre_fma"] += cnt * head["fma"]
            tot["pre_mul"] += cnt * head["mul"]
            for v in range(u + 1, n - D):
                tot["pre_fma"] += cnt * ext["fma"]
                tot["pre_mul"] += cnt * ext["mul"]
                tot["upd_fma"] += cnt * D * H
                body(cnt, n - 1 - v)
    else:
        for v in range(P - 1, n - D):
            cnt = math.comb(v, P - 1)
            tot["pre_fma"] += cnt * pre["fma"]
            tot["pre_mul"] += cnt * pre["mul"]
            body(cnt, n - 1 - v)
    tot["all_fma"] = tot["pre_fma"] + tot["fma"]
    tot["all_mul"] = tot["pre_mul"] + tot["mul"]
    tot["all_add"] = tot["add"]
    return tot


def prefix_flops(m: int, n: int, D: int) -> int:
    """Algorithmic flops of the prefix path in one arithmetic: 2 per FMA, 1 per add or multiply."""
    c = prefix_ops(m, n, D)
    return 2 * c["all_fma"] + c["all_mul"] + c["all_add"]


# binary32 flops of the pair algorithms (radic_ff.cuh): multiply-add 18
# (exact product 7, TwoSum 6, low parts 2, Fast2Sum 3), multiply 10, addition
# 11; the magnitude sum of the leaves stays one binary32 addition per leaf
PAIR_FMA, PAIR_MUL, PAIR_ADD = 18, 10, 11


def pair_flops(m: int, n: int, D: int, shared: bool = False) -> dict:
    """The pair tier's work: binary32 flops (pair algorithms) of the columns,
    column pairs and leaves, and with head sharing of the extensions' W
    updates, on the binary32 pipe; the binary64 flops of the rest of the
    prefix factorisations (heads, extensions) on the binary64 pipe."""
    c = prefix_ops(m, n, D, shared)
    leaves = c["add"] // 2
    return {"fp32": PAIR_FMA * (c["fma"] + c["upd_fma"]) + PAIR_MUL * c["mul"] + PAIR_ADD * leaves + leaves,
            "fp64": 2 * (c["pre_fma"] - c["upd_fma"]) + c["pre_mul"]}


def modp_mults(m: int, n: int, D: int, primes: int) -> int:
    """32-bit integer multiplies of the exact prefix path (radic_modp_prefix.cu)
    for all C(n,m) minors: a fraction-free update (a_kk a_ij - a_ik a_kj,
    Montgomery-reduced) is 4 multiplies, a Montgomery product 3, a reduction
    2, a leaf dot product (D = 3) 7.  Per prefix and prime: the elimination of
    its m x P block and the P pivots' products (2P + D - 1 products); per
    candidate column: its elimination (sum_k (m-1-k) updates) and the
    column-sum conversion (a reduction and a product); per column pair (D = 3)
    a cross product (3 updates); per leaf a dot product (D = 3) or a 2 x 2
    update (D = 2); per prefix the fraction update (3 products)."""
    P = m - D
    per_pre = 4 * sum((m - 1 - k) * (P - 1 - k) for k in range(P)) + 3 * (2 * P + D - 1) + 3 * 3
    per_col = 4 * sum(m - 1 - k for k in range(P)) + 2 + 3
    per_pair = 12 if D == 3 else 0
    per_leaf = 7 if D == 3 else 4
    tot = 0
    for v in range(P - 1, n - D):
        cnt = math.comb(v, P - 1)
        k = n - 1 - v
        tot += cnt * (per_pre + k * per_col + math.comb(k, 2) * per_pair + math.comb(k, D) * per_leaf)
    return tot * primes


# ---------------------------------------------------------------------------
# oracle baseline (CPU, spawn pool)
# ---------------------------------------------------------------------------
def _oracle_chunk(args):
    """Exact minors of Eq. (1) (the oracle's Bareiss enumeration) for ranks [lo, hi) of one matrix."""
    lo, hi, name, index = args
    sys.path.insert(0, ROOT)
    import oracle.radic_oracle as orc
    from paper_1508_01326_gb300 import workloads as W

    if name == "batched_4096":
        a = W.batched_4096()[index]
    elif name == "int_3x12":
        a = W.int_3x12()
    elif name == "int8_10x24":
        a = W.int8_10x24()
    elif name == "diff_6x28":
        a = W.diff_256x6x28()[0]
    else:
        a = W.fp64_8x32()
    terms = orc.radic_terms_exact(a, range(lo, hi))
    return hi - lo, float(sum(terms))


def oracle_rate(pool, cores: int, sample: int, offset: int, name: str, index: int = 0) -> float:
    per = -(-sample // cores)
    chunks = [(offset + i * per, min(offset + (i + 1) * per, offset + sample), name, index) for i in range(cores)]
    chunks = [c for c in chunks if c[0] < c[1]]
    t0 = time.perf_counter()
    done = sum(n for n, _ in pool.map(_oracle_chunk, chunks))
    return done / (time.perf_counter() - t0)


def make_pool():
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(cores)
    pool.map(_oracle_chunk, [(0, 1, "fp64_8x32", 0)] * cores)  # import the oracle in every worker before timing
    return pool, cores


# the batch matrices whose ranks the oracle samples: the largest of each m (m >= 3)
def _oracle_batch_sample():
    from paper_1508_01326_gb300 import workloads as W

    mats = W.batched_4096()
    pick = {}
    for i, a in enumerate(mats):
        m, n = a.shape
        if 3 <= m <= n and (m not in pick or math.comb(n, m) > math.comb(*mats[pick[m]].shape[::-1])):
            pick[m] = i
    return [pick[m] for m in sorted(pick)]


def oracle_batch_rate(pool, cores: int, per_matrix: int) -> tuple:
    """Exact-oracle minors per second on `per_matrix` consecutive ranks of the largest matrix of each
    m of the batch (ranks from the middle of the matrix's range)."""
    from paper_1508_01326_gb300 import workloads as W

    mats = W.batched_4096()
    chunks = []
    for i in _oracle_batch_sample():
        m, n = mats[i].shape
        total = math.comb(n, m)
        q0 = max(0, total // 2 - per_matrix // 2)
        cnt = min(per_matrix, total - q0)
        per = -(-cnt // cores)
        chunks += [(q0 + j * per, min(q0 + (j + 1) * per, q0 + cnt), "batched_4096", i) for j in range(cores)
                   if q0 + j * per < q0 + cnt]
    t0 = time.perf_counter()
    done = sum(n for n, _ in pool.map(_oracle_chunk, chunks))
    return done / (time.perf_counter() - t0), done


def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    pool, cores = make_pool()
    per_matrix = 2 * cores * 40
    try:
        for _ in range(args.warmup):
            oracle_batch_rate(pool, cores, per_matrix)
        t0 = time.perf_counter()
        done = 0
        for _ in range(args.steps):
            done += oracle_batch_rate(pool, cores, per_matrix)[1]
        dt = time.perf_counter() - t0
    finally:
        pool.terminate()
    value = done / dt
    desc = (f"exact Bareiss minors of Eq. (1) (the oracle) for {per_matrix} consecutive dictionary ranks of the "
            f"largest matrix of each m = 3..10 of the batch per step, over {cores} spawn workers")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "exact", "data": "synthetic",
        "config": {"workload": WORKLOAD, "mode": "oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def max_over_ranks(total_ms: float, device=None) -> float:
    """Slowest rank's timed total (all ranks call it; a no-op without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return total_ms
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measure_peaks(torch, stream, sampler_factory) -> dict:
    """Pipe peaks measured with the FMA-chain probe (libradic_peaks.so) at the clocks of this run:
    binary32 and binary64 FMA (TFLOP/s, 2 flop per FMA) and 32-bit and 32x32->64-bit integer
    multiply-add (T operations/s); each about 0.1-0.3 s, with the SM clock sampled meanwhile."""
    from paper_1508_01326_gb300 import build as B

    L = ctypes.CDLL(B.PEAKS_LIB_PATH)
    L.radic_peak_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.radic_peak_probe.restype = ctypes.c_int
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    scratch = torch.empty(8 * sms * 256 * 8, dtype=torch.uint8, device="cuda")
    out = {}
    sampler = sampler_factory()
    sampler.start()
    for name, kind, iters, scale in [("fp32_tflops", 0, 6000, 2.0), ("fp64_tflops", 1, 150, 2.0),
                                     ("int32_mad_tops", 2, 3000, 1.0), ("int32_mad_wide_tops", 3, 3000, 1.0)]:
        best = 0.0
        for _ in range(3):
            ops, ms = ctypes.c_double(), ctypes.c_double()
            rc = L.radic_peak_probe(kind, 8, iters, scratch.data_ptr(), stream.cuda_stream, ctypes.byref(ops),
                                    ctypes.byref(ms))
            if rc != 0:
                raise RuntimeError(f"radic_peak_probe({kind}) failed: {rc}")
            best = max(best, ops.value * scale / 1e12)
        out[name] = best
    out["clocks"] = sampler.stop()
    out["how"] = ("best of 3 launches of 8 blocks x 256 threads per SM, 8 independent chains of one operation per "
                  "thread (libradic_peaks.so); FMA counted as 2 flop, integer multiply-add as 1 operation")
    return out


def run_ours(args, rank: int, world: int, local_rank: int) -> None:
    import numpy as np
    import torch

    pool = None
    cores = 0
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool, cores = make_pool()  # spawn context: safe to start before CUDA

    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_1508_01326_gb300 import autotune
    from paper_1508_01326_gb300 import build as B

    B.build()
    import paper_1508_01326_gb300 as R
    from paper_1508_01326_gb300 import workloads as W

    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2

    peaks = measure_peaks(torch, stream, lambda: ClockSampler(local_rank)) if rank == 0 else None

    # ---- headline: the 4096-matrix batch through the MIXED router -------------------------------
    mats = W.batched_4096()
    minors = sum(math.comb(x.shape[1], x.shape[0]) for x in mats if x.shape[0] <= x.shape[1])
    gold = golden_values("batched_4096_f64")
    scale = golden_abs_sums("batched_4096_f64")
    data, ms_, ns_, offs = W.pack_batch(mats, np.float64)
    A = torch.from_numpy(data).cuda()
    tuning, table = autotune.autotune(mats, mode="mixed", tol=TOL)
    kev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for e in kev:
        e.record(stream)  # create the underlying events
    handles = (ctypes.c_void_p * 2)(kev[0].cuda_event, kev[1].cuda_event)
    tuning.kernel_events = ctypes.addressof(handles)
    plan = R.BatchPlan(list(zip(ms_, ns_)), offs, mode="mixed", tuning=tuning)
    info = plan.info()
    out = plan.new_results()
    graph = plan.graph(A, out)

    def step():
        flush.zero_()  # untimed: the L2 holds nothing of the batch when a step starts
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.launch(stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), kev[0].elapsed_time(kev[1])

    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(local_rank)
    sampler.start()
    t_end = time.time() + args.settle_seconds
    while time.time() < t_end:
        graph.launch(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms, kern_ms = [], []
    for _ in range(args.steps):
        s_ms, k_ms = step()
        step_ms.append(s_ms)
        kern_ms.append(k_ms)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(step_ms), device="cuda")
    ms_per_step = total_ms / args.steps
    value = world * minors / (ms_per_step / 1e3)

    rs = R.parse_results(out)
    rel = [abs(r["value"] - w) / s for r, w, s in zip(rs, gold, scale) if s > 0]
    bnd = [r["err_bound"] / s for r, s in zip(rs, scale) if s > 0]
    held = all(abs(r["value"] - w) <= r["err_bound"] + 0.5 * math.ulp(w) for r, w, s in zip(rs, gold, scale) if s > 0)
    tiers = {}
    for r in rs:
        tiers[r["tier"]] = tiers.get(r["tier"], 0) + 1

    # roofline of the dominant kernel: its group's algorithmic work over its event time
    dm, dpath = info["dominant_m"], info["dominant_path"]
    D = {1: 2, 2: 3, 3: 2, 4: 3}.get(dpath, 0)
    shared = dpath in (3, 4)
    dom_fp32 = dom_fp64 = 0
    dom_matrices = 0
    for a in mats:
        mm, nn = a.shape
        if mm == dm and mm <= nn and D:
            dflt = 3 if mm >= 6 and 2 * (nn - mm) <= 7 * mm else 2
            v = table.get(str(mm), table.get(mm, {}))
            if (v.get("depth") or dflt) == D:
                f = pair_flops(mm, nn, D, shared)
                dom_fp32 += f["fp32"]
                dom_fp64 += f["fp64"]
                dom_matrices += 1
    kern_mean = statistics.mean(kern_ms)
    achieved = dom_fp32 / (kern_mean / 1e3) / 1e12
    fp32_peak = peaks["fp32_tflops"] if peaks else None
    path_name = {0: "per-minor", 1: "prefix depth 2", 2: "prefix depth 3", 3: "head-shared depth 2",
                 4: "head-shared depth 3"}[dpath]
    roofline = {
        "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
        "frac": achieved / fp32_peak if fp32_peak else None, "traffic": DOMINANT_DRAM_BYTES,
        "kernel": f"k_batch<ff,1,{dm},{dpath}> (pair tier, m = {dm}, {path_name})",
        "kernel_ms": kern_mean, "matrices": dom_matrices,
        "flop_per_launch": dom_fp32, "fp64_flop_per_launch": dom_fp64,
        "fp64_frac": dom_fp64 / (kern_mean / 1e3) / 1e12 / peaks["fp64_tflops"] if peaks else None,
        "peak_source": "measured: binary32 FMA-chain probe in this run (libradic_peaks.so), 2 flop per FMA",
        "flop_rule": ("binary32 flops of the pair algorithms for the Schur-complement columns, column pairs and "
                      "leaves (multiply-add 18, multiply 10, addition 11 + 1 for the magnitude sum); the prefix "
                      "factorisations run in binary64 and are reported as fp64_flop_per_launch"),
    }
    # the whole step: every pair-tier matrix's algorithmic work over the step time (the per-group
    # kernels of a phase run concurrently, so the dominant kernel's own span also holds the others' tails)
    step_fp32 = step_fp64 = 0
    for a, r in zip(mats, rs):
        mm, nn = a.shape
        if r["tier"] != 3 or mm > nn or mm < 3:
            continue
        dflt = 3 if mm >= 6 and 2 * (nn - mm) <= 7 * mm else 2
        v = table.get(str(mm), table.get(mm, {}))
        dd = v.get("depth") or dflt
        f = pair_flops(mm, nn, dd, mm - dd - 1 >= 5)
        step_fp32 += f["fp32"]
        step_fp64 += f["fp64"]
    step_achieved = step_fp32 / (ms_per_step / 1e3) / 1e12
    roofline["step"] = {
        "achieved": step_achieved, "frac": step_achieved / fp32_peak if fp32_peak else None,
        "fp64_frac": step_fp64 / (ms_per_step / 1e3) / 1e12 / peaks["fp64_tflops"] if peaks else None,
        "flop": step_fp32, "fp64_flop": step_fp64,
        "rule": "binary32 flops of every pair-tier matrix (same rule) over ms_per_step"}
    headline_tiers = {"binary64": tiers.get(0, 0), "binary32": tiers.get(1, 0), "pairs": tiers.get(3, 0)}

    configs = None
    if rank == 0 and not args.headline_only:
        configs = measure_configs(R, W, torch, np, stream, flush, peaks, mats, A, minors, gold, scale)

    # ---- end to end: pinned host input, the public batched call, results back to the host ---------
    a_host = torch.from_numpy(data).pin_memory()
    res_host = torch.empty_like(out, device="cpu").pin_memory()
    a_dev = torch.empty_like(A)
    plan_e2e = R.BatchPlan(list(zip(ms_, ns_)), offs, mode="mixed", tuning=autotune.autotune(mats, "mixed", TOL)[0])
    out_e2e = plan_e2e.new_results()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        a_dev.copy_(a_host, non_blocking=True)
        plan_e2e.radic_det_batched(a_dev, out_e2e, stream=stream)
        res_host.copy_(out_e2e, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if i >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_rate = world * minors / (statistics.mean(e2e_ms) / 1e3)
    plan_e2e.close()

    cpu = None
    if pool is not None:
        rate, done = oracle_batch_rate(pool, cores, 2 * cores * 60)
        oracle_configs = {
            "fp64_8x32": {"value": oracle_rate(pool, cores, 80_000, ORACLE_SAMPLE_OFFSET, "fp64_8x32"),
                          "sample": "80,000 ranks from rank 1,000,000"},
            "int8_10x24": {"value": oracle_rate(pool, cores, 40_000, 500_000, "int8_10x24"),
                           "sample": "40,000 ranks from rank 500,000 of the 10x24 subcase"},
            "diff_6x28": {"value": oracle_rate(pool, cores, 40_000, 100_000, "diff_6x28"),
                          "sample": "40,000 ranks from rank 100,000 of the first 6x28 matrix"}}
        pool.terminate()
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": (f"exact Bareiss minors of Eq. (1) for {done} dictionary ranks: {2 * cores * 60} "
                          f"consecutive ranks from the middle of the largest matrix of each m = 3..10 of the "
                          f"same batch, over {cores} spawn workers"),
               "oracle_configs": oracle_configs,
               "fp64_enumeration": cpu_enumeration_rates(W, np)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "pair-f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "matrices": len(mats), "minors": minors, "mode": "mixed",
                       "tol": TOL, "routing": info, "final_tiers": headline_tiers,
                       "autotune": {m: v["kind"] + (str(v["depth"]) if v.get("depth") else "") + "/" +
                                    str(int(v["task_cost"])) for m, v in table.items()},
                       "l2": "flushed between timed iterations (256 MB write, untimed)",
                       "launch": "each step replays a CUDA graph of one radic_det_batched call",
                       "parallelism": f"replicas{world}"},
            "rel_err_max": max(rel), "err_bound_max": max(bnd), "bound_held": held,
            "roofline": roofline,
            "peaks": peaks,
            "clocks": clocks,
            "configs": configs,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_rate, "unit": UNIT, "h2d_bytes_per_step": int(A.numel() * 8),
                    "d2h_bytes_per_step": int(out.numel() * 8)},
            "gpu_launches": int(info["launches"]) * args.steps,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_enumeration_rates(W, np) -> dict:
    """The binary64 host enumeration of Eq. (1) (oracle/radic_cpu.c: Section 5 runs over OpenMP
    threads, partial-pivot LU per minor) on every configuration, at full size where it takes
    seconds and on stated samples elsewhere; minors per second."""
    from oracle import cpu_enum

    def rate(mats, counts=None, q0s=None):
        done, t0, th = 0, time.perf_counter(), 1
        for i, a in enumerate(mats):
            q0 = q0s[i] if q0s else 0
            cnt = counts[i] if counts else math.comb(a.shape[1], a.shape[0])
            _, _, th = cpu_enum.radic_cpu_sum(a, q0, cnt)
            done += cnt
        return done / (time.perf_counter() - t0), th, done

    out = {}
    sub = W.batched_4096()[::64]
    r, th, done = rate(sub)
    out["batched_4096"] = {"value": r, "minors": done, "sample": "every 64th matrix (64 matrices), full"}
    r, th, done = rate([W.fp64_8x32()])
    out["fp64_8x32"] = {"value": r, "minors": done, "sample": "full"}
    r, th, done = rate([W.int8_12x40().astype(np.float64)], counts=[20_000_000], q0s=[1_000_000_000])
    out["int8_12x40"] = {"value": r, "minors": done, "sample": "20,000,000 ranks from rank 1e9 (binary64, not exact)"}
    r, th, done = rate(list(W.diff_256x6x28()[:8]))
    out["diff_256x6x28"] = {"value": r, "minors": done, "sample": "first 8 matrices (forward only), full"}
    out["threads"] = th
    out["unit"] = UNIT
    return out


def measure_configs(R, W, torch, np, stream, flush, peaks, mats, A, minors, gold, scale) -> dict:
    """The other configurations and comparison paths (not the headline)."""
    def ev_time(fn, reps=1, flush_l2=True):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            if flush_l2:
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    out = {}
    # the batch through the plain binary64 batched path, and one plain binary64 launch per matrix
    plan = R.BatchPlan([x.shape for x in mats], None, mode="fp64")
    o = plan.new_results()
    g = plan.graph(A, o)
    ms = ev_time(g.launch, reps=3)
    rs = R.parse_results(o)
    out["batched_4096_fp64"] = {
        "value": minors / (ms / 1e3), "unit": UNIT, "ms": ms,
        "rel_err_max": max(abs(r["value"] - w) / s for r, w, s in zip(rs, gold, scale) if s > 0),
        "err_bound_max": max(r["err_bound"] / s for r, s in zip(rs, scale) if s > 0)}
    plan.close()
    dev = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in mats]
    outs = R.new_result().new_empty((len(mats), 16))
    wss = [torch.empty(max(R.radic_workspace_bytes(x.shape[0], x.shape[1], "fp64",
                                                   dict(mapping="thread" if x.shape[0] <= 8 else "group")), 256),
                       dtype=torch.uint8, device="cuda") for x in mats]

    def per_matrix():
        for i, x in enumerate(dev):
            R.radic_det(x, mode="fp64", options=dict(mapping="thread" if x.shape[0] <= 8 else "group"),
                        out=outs[i], workspace=wss[i])

    ms = ev_time(per_matrix, reps=1)
    rs = R.parse_results(outs)
    out["per_matrix_plain_fp64"] = {
        "value": minors / (ms / 1e3), "unit": UNIT, "ms": ms, "launches": 2 * len(mats),
        "rel_err_max": max(abs(r["value"] - w) / s for r, w, s in zip(rs, gold, scale) if s > 0),
        "what": "one radic_det per matrix, per-minor binary64 LU (thread mapping, warp groups for m > 8)"}

    # 8 x 32 single matrix in every mode (graph replay of one radic_det call)
    a = torch.from_numpy(W.fp64_8x32()).cuda()
    exact = golden_values("fp64_8x32")[0]
    s32 = golden_abs_sums("fp64_8x32")[0]
    single = {}
    for mode, mapping in [("mixed", "auto"), ("pair", "auto"), ("fp64", "auto"), ("fp64", "thread"),
                          ("mixed", "thread")]:
        res = R.new_result()
        ws = torch.empty(R.radic_workspace_bytes(8, 32, mode, dict(mapping=mapping)), dtype=torch.uint8,
                         device="cuda")
        R.radic_det(a, mode=mode, options=dict(mapping=mapping), out=res, workspace=ws)
        gr = R.DetGraph(a, mode=mode, options=dict(mapping=mapping), out=res, workspace=ws)
        ms = ev_time(lambda: gr.launch(stream), reps=10)
        r = R.parse_result(res)
        single[f"{mode}/{mapping}"] = {"value": math.comb(32, 8) / (ms / 1e3), "unit": UNIT, "ms": ms,
                                       "rel_err": abs(r["value"] - exact) / s32, "err_bound": r["err_bound"] / s32,
                                       "flagged": r["flagged"]}
    out["fp64_8x32"] = single

    # exact 3 x 12 int32: latency of one call
    a = torch.from_numpy(W.int_3x12()).cuda()
    res = R.new_result()
    ws = torch.empty(R.radic_workspace_bytes(3, 12, "exact"), dtype=torch.uint8, device="cuda")
    ms = ev_time(lambda: R.radic_det(a, mode="exact", out=res, workspace=ws), reps=50, flush_l2=False)
    out["int_3x12_exact"] = {"us_per_call": ms * 1e3,
                             "exact_ok": R.parse_result(res)["exact"] == int(golden_fraction("int_3x12"))}
    # exact 12 x 40 int8: full size, with the integer-multiply roofline
    a = torch.from_numpy(W.int8_12x40()).cuda()
    ws = torch.empty(R.radic_workspace_bytes(12, 40, "exact"), dtype=torch.uint8, device="cuda")
    ms = ev_time(lambda: R.radic_det(a, mode="exact", out=res, workspace=ws), reps=3)
    r = R.parse_result(res)
    pinfo = R.radic_plan_info(12, 40, "exact")
    mults = modp_mults(12, 40, pinfo["prefix_depth"], r["n_primes"])
    mult_rate = mults / (ms / 1e3) / 1e12
    out["int8_12x40_exact"] = {
        "value": r["minors"] / (ms / 1e3), "unit": UNIT, "ms": ms, "n_primes": r["n_primes"],
        "exact_ok": r["exact"] == int(golden_fraction("int8_12x40")),
        "mapping": f"{pinfo['mapping']} depth {pinfo['prefix_depth']}",
        "roofline": {"bound": "alu", "achieved": mult_rate, "unit": "T multiplies/s",
                     "peak": peaks["int32_mad_wide_tops"] if peaks else None,
                     "frac": mult_rate / peaks["int32_mad_wide_tops"] if peaks else None,
                     "work": mults, "peak_source": "measured: 32x32->64-bit multiply-add chain probe in this run"}}

    # exact 8 x 32 binary64 (rows scaled to integers, beyond 128 bits): wide exact mode
    a = torch.from_numpy(W.fp64_8x32()).cuda()
    wres = torch.zeros(R.api.WIDE_RESULT_BYTES, dtype=torch.uint8, device="cuda")
    wws = torch.empty(int(R._lib.lib().radic_wide_workspace_bytes(8, 32, None)), dtype=torch.uint8, device="cuda")
    ms = ev_time(lambda: R.radic_det_exact_wide(a, out=wres, workspace=wws), reps=3)
    wr = R.parse_wide_result(wres)
    out["fp64_8x32_exact_wide"] = {
        "value": math.comb(32, 8) / (ms / 1e3), "unit": UNIT, "ms": ms, "n_primes": wr["n_primes"],
        "bits": abs(wr["integer"]).bit_length(),
        "exact_ok": wr["value_exact"] == golden_fraction("fp64_8x32"),
        "what": "radic_det_exact_wide: RADIC_MAX_PRIMES primes per pass of the exact kernels, Garner to limbs"}

    # differentiation 256 x 6 x 28: forward (batched binary64) and backward
    Dm = torch.from_numpy(W.diff_256x6x28()).cuda()
    g_out = torch.ones(256, dtype=torch.float64, device="cuda")
    fwd = ev_time(lambda: R.RadicDet.apply(Dm), reps=3)
    bwd = ev_time(lambda: R.radic_det_backward(Dm, g_out), reps=3)
    mn = 256 * math.comb(28, 6)
    out["diff_256x6x28"] = {"forward_ms": fwd, "backward_ms": bwd, "backward_minors_per_s": mn / (bwd / 1e3),
                            "forward_minors_per_s": mn / (fwd / 1e3)}
    fwd_m = ev_time(lambda: R.RadicDet.apply(Dm, "mixed"), reps=3)
    bwd_m = ev_time(lambda: R.radic_det_backward(Dm, g_out, mode="pair"), reps=3)
    out["diff_256x6x28"]["mixed"] = {"forward_ms": fwd_m, "backward_ms": bwd_m,
                                     "backward_minors_per_s": mn / (bwd_m / 1e3)}
    return out


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--settle-seconds", type=float, default=1.0)
    ap.add_argument("--headline-only", action="store_true", help="skip the other configurations")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.gpus == 1 else 1)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
