"""Command-line runner: one workload, one mode, a few repetitions.

    python -m paper_1508_01326_gb300.cli --workload fp64_8x32 --mode mixed --reps 3

Prints the parsed result and the CUDA-event time of each repetition.  Useful
as a small, self-contained target for profilers.
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


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="fp64_8x32", choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default="mixed", choices=["fp64", "mixed", "exact"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--mapping", default="auto", choices=["auto", "thread", "group", "prefix"])
    ap.add_argument("--group-width", type=int, default=0)
    ap.add_argument("--ranks-per-task", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    from . import build as B

    B.build()
    a = torch.from_numpy(np.ascontiguousarray(WORKLOADS[args.workload]())).cuda()
    opts = dict(mapping=args.mapping, group_width=args.group_width, ranks_per_task=args.ranks_per_task,
                threads_per_block=args.threads)
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
