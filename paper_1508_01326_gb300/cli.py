"""Command-line runner: one workload, one mode, a few repetitions.

    python -m paper_1508_01326_gb300.cli --workload fp64_8x32 --mode mixed --reps 3
    python -m paper_1508_01326_gb300.cli --batched-m 10 --mode mixed --tol 1e-10 --reps 2
    python -m paper_1508_01326_gb300.cli --backward --batch 32 --mode fp64 --reps 1

Prints the parsed result and the CUDA-event time of each repetition.  Useful
as a small, self-contained target for profilers.  With --batched-m the run
is the batched path over the matrices with that m of the 4096-matrix batch;
with --backward it is the gradient kernel over the first --batch matrices of
the 256 x 6 x 28 workload with grad_out = 1.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import api
from . import workloads as W

WORKLOADS = {
    "int_3x12": W.int_3x12,
    "fp64_8x32": W.fp64_8x32,
    "fp32_8x32": lambda: W.fp64_8x32().astype(np.float32),
    "int8_10x24": W.int8_10x24,
    "int8_12x40": W.int8_12x40,
    "diff_6x28": lambda: W.diff_256x6x28()[0],
}


def run_batched(args) -> None:
    mats = [a for a in W.batched_4096() if a.shape[0] == args.batched_m]
    data, ms, ns, offs = W.pack_batch(mats, np.float64)
    A = torch.from_numpy(data).cuda()
    depth = {args.batched_m: args.depth} if args.depth else None
    tuning = api.make_tuning(tol=args.tol, prefix_depth=depth)
    plan = api.BatchPlan(list(zip(ms, ns)), offs, mode=args.mode, tuning=tuning)
    out = plan.new_results()
    times = []
    for _ in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.radic_det_batched(A, out)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    print(json.dumps({"batched_m": args.batched_m, "matrices": len(mats), "mode": args.mode, "ms": times,
                      "routing": plan.info()}))
    plan.close()


def run_backward(args) -> None:
    from .autograd import radic_det_backward

    A = torch.from_numpy(np.ascontiguousarray(W.diff_256x6x28()[: args.batch])).cuda()
    g = torch.ones(A.shape[0], dtype=torch.float64, device="cuda")
    mode = args.mode if args.mode in ("fp64", "pair") else "fp64"
    times = []
    for _ in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        grad = radic_det_backward(A, g, mode=mode)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    print(json.dumps({"backward": list(A.shape), "mode": mode, "ms": times,
                      "grad_abs_max": float(grad.abs().max().item())}))


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="fp64_8x32", choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default="mixed", choices=["fp64", "mixed", "exact", "pair"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--mapping", default="auto", choices=["auto", "thread", "group", "prefix"])
    ap.add_argument("--group-width", type=int, default=0)
    ap.add_argument("--ranks-per-task", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--depth", type=int, default=0, help="prefix depth (0: library default)")
    ap.add_argument("--batched-m", type=int, default=0, help="batched path over this m of the 4096 batch")
    ap.add_argument("--tol", type=float, default=1e-10, help="batched MIXED router tolerance")
    ap.add_argument("--backward", action="store_true", help="gradient kernel over the 6 x 28 workload")
    ap.add_argument("--batch", type=int, default=32, help="matrices of the 256 x 6 x 28 workload (--backward)")
    args = ap.parse_args()
    from . import build as B

    B.build()
    if args.backward:
        run_backward(args)
        return
    if args.batched_m:
        run_batched(args)
        return
    a = torch.from_numpy(np.ascontiguousarray(WORKLOADS[args.workload]())).cuda()
    opts = dict(mapping=args.mapping, group_width=args.group_width, ranks_per_task=args.ranks_per_task,
                threads_per_block=args.threads, prefix_depth=args.depth)
    out = api.new_result()
    ws = torch.empty(max(api.radic_workspace_bytes(*a.shape, mode=args.mode, options=opts), 256),
                     dtype=torch.uint8, device="cuda")
    times = []
    for _ in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        api.radic_det(a, mode=args.mode, options=opts, out=out, workspace=ws)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    res = api.parse_result(out)
    res["exact"] = str(res["exact"])
    print(json.dumps({"workload": args.workload, "mode": args.mode, "ms": times, "result": res}))


if __name__ == "__main__":
    main()
