"""Python binding of the C ABI (include/radic.h): same entry-point names, torch
tensors in and out.  PyTorch supplies device memory and streams only; every
step of the computation runs in libradic.so.  There is no CPU fallback: when
the library is missing or CUDA is unavailable these functions raise.
"""
from __future__ import annotations

import ctypes
import struct
from fractions import Fraction
from typing import Optional

import numpy as np
import torch

from . import _lib as L

_TORCH_DTYPES = {torch.int8: 0, torch.int32: 1, torch.float32: 2, torch.float64: 3}
_NP_TO_TORCH = {np.dtype(np.int8): torch.int8, np.dtype(np.int32): torch.int32,
                np.dtype(np.float32): torch.float32, np.dtype(np.float64): torch.float64}


def _mode(mode) -> int:
    return L.MODES[mode] if isinstance(mode, str) else int(mode)


def _opts(options) -> Optional[ctypes.POINTER(L.RadicOptions)]:
    if options is None:
        return None
    if isinstance(options, dict):
        options = L.make_options(**options)
    return ctypes.pointer(options)


def _stream(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check_matrix(A: torch.Tensor) -> None:
    if not isinstance(A, torch.Tensor) or not A.is_cuda:
        raise TypeError("A must be a CUDA tensor")
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be a 2-D row-major tensor with unit column stride")
    if A.dtype not in _TORCH_DTYPES:
        raise TypeError(f"unsupported dtype {A.dtype}")


def radic_status_string(code: int) -> str:
    return L.lib().radic_status_string(int(code)).decode()


def radic_version() -> int:
    return L.lib().radic_version()


def radic_primes() -> list:
    buf = (ctypes.c_uint32 * L.RADIC_MAX_PRIMES)()
    k = L.lib().radic_primes(buf, L.RADIC_MAX_PRIMES)
    return [int(buf[i]) for i in range(k)]


def radic_workspace_bytes(m: int, n: int, mode="fp64", options=None) -> int:
    return int(L.lib().radic_workspace_bytes(int(m), int(n), _mode(mode), _opts(options)))


PLAN_INFO_KEYS = ["mapping", "prefix_depth", "group_width", "threads", "blocks", "run_or_tasks", "smem_bytes",
                  "workspace_bytes"]
MAPPING_NAMES = {1: "thread", 2: "group", 3: "prefix"}


def radic_plan_info(m: int, n: int, mode="fp64", options=None) -> dict:
    """The launch plan radic_det would use (host only, no launch)."""
    buf = (ctypes.c_int64 * len(PLAN_INFO_KEYS))()
    opts = _opts(options)
    L.check("radic_plan_info", L.lib().radic_plan_info(int(m), int(n), _mode(mode), opts, buf, len(buf)))
    info = dict(zip(PLAN_INFO_KEYS, [int(x) for x in buf]))
    info["mapping"] = MAPPING_NAMES.get(info["mapping"], info["mapping"])
    return info


def prefix_plan_host(m: int, n: int, mode="mixed", options=None, sms: int = 152, blocks_per_sm: int = 3) -> dict:
    """The prefix mapping's task table for a given SM count and residency, planned on the host
    only (radic_prefix_plan_host): depth, tasks, blocks, and per last prefix column v the prefix
    count, run length, lanes per prefix and first task."""
    count = 8 + 4 * int(n)
    buf = (ctypes.c_int64 * count)()
    L.check("radic_prefix_plan_host", L.lib().radic_prefix_plan_host(int(m), int(n), _mode(mode), _opts(options),
                                                                     int(sms), int(blocks_per_sm), buf, count))
    v_lo, v_hi = int(buf[3]), int(buf[4])
    groups = {v: {"count": int(buf[8 + 4 * v]), "run": int(buf[9 + 4 * v]), "lanes": int(buf[10 + 4 * v]),
                  "task_start": int(buf[11 + 4 * v])} for v in range(v_lo, v_hi + 1)}
    return {"depth": int(buf[0]), "tasks": int(buf[1]), "blocks": int(buf[2]), "v_lo": v_lo, "v_hi": v_hi,
            "dynamic": bool(buf[5]), "groups": groups}


def new_result(device=None) -> torch.Tensor:
    """Device buffer for one radic_result (sixteen int64 words)."""
    return torch.empty(L.RESULT_WORDS, dtype=torch.int64, device=device or "cuda")


def radic_det(A: torch.Tensor, mode="fp64", options=None, out: Optional[torch.Tensor] = None,
              workspace: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Enqueues det_R(A) on `stream`; returns the device result buffer (not synchronised)."""
    _check_matrix(A)
    m, n = A.shape
    md = _mode(mode)
    lib = L.lib()
    if out is None:
        out = new_result(A.device)
    ws_bytes = int(lib.radic_workspace_bytes(int(m), int(n), md, _opts(options)))
    if workspace is None:
        workspace = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=A.device)
    rc = lib.radic_det(A.data_ptr(), int(m), int(n), int(A.stride(0)), _TORCH_DTYPES[A.dtype], md, _opts(options),
                       out.data_ptr(), workspace.data_ptr(), workspace.numel(), _stream(stream))
    L.check("radic_det", rc)
    return out


def radic_terms(A: torch.Tensor, q0: int, count: int, mode="fp64", options=None,
                out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Signed terms of Eq. (1) for dictionary ranks q0 .. q0+count-1 (device tensor)."""
    _check_matrix(A)
    m, n = A.shape
    md = _mode(mode)
    if out is None:
        if md == L.MODES["exact"]:
            out = torch.zeros((L.RADIC_MAX_PRIMES, max(int(count), 1)), dtype=torch.int32, device=A.device)
        else:
            out = torch.empty(max(int(count), 1), dtype=torch.float64, device=A.device)
    rc = L.lib().radic_terms(A.data_ptr(), int(m), int(n), int(A.stride(0)), _TORCH_DTYPES[A.dtype], md,
                             _opts(options), int(q0), int(count), out.data_ptr(), _stream(stream))
    L.check("radic_terms", rc)
    return out


def radic_unrank(n: int, m: int, q0: int, count: int, options=None, out: Optional[torch.Tensor] = None,
                 stream=None, device="cuda") -> torch.Tensor:
    """Column sequences (0-based) of dictionary ranks q0 .. q0+count-1, shape (count, m), uint8."""
    if out is None:
        out = torch.empty((max(int(count), 1), int(m)), dtype=torch.uint8, device=device)
    rc = L.lib().radic_unrank(int(n), int(m), int(q0), int(count), out.data_ptr(), _opts(options), _stream(stream))
    L.check("radic_unrank", rc)
    return out


def parse_result(buf: torch.Tensor) -> dict:
    """Host dictionary of a radic_result buffer (copies it to the host)."""
    w = buf.detach().to("cpu").contiguous()
    f = w.view(torch.float64)
    lo = int(w[3]) & ((1 << 64) - 1)
    hi = int(w[4])
    exact = (hi << 64) | lo
    return {
        "value": float(f[0]),
        "abs_sum": float(f[1]),
        "err_bound": float(f[2]),
        "exact": exact,
        "minors": int(w[5]),
        "flagged": int(w[6]),
        "status": int(w[7]),
        "n_primes": int(w[8]),
        "tier": int(w[9]),
        "exact_exp": int(w[10]),
    }


def det(A, mode="fp64", options=None, stream=None) -> dict:
    """Convenience call: host (numpy) or device input, synchronises and returns a dict.

    A host array is copied to the device first (this is the end-to-end path).
    """
    if isinstance(A, np.ndarray):
        A = torch.from_numpy(np.ascontiguousarray(A)).to("cuda")
    out = radic_det(A, mode=mode, options=options, stream=stream)
    res = parse_result(out)
    if res["status"] != 0:
        raise L.RadicError("radic_det (device)", res["status"])
    if _mode(mode) == L.MODES["exact"]:
        # det_R(A) = exact * 2^exact_exp (the exponent is 0 for integer inputs)
        e = res["exact_exp"]
        res["value_exact"] = Fraction(res["exact"]) * (Fraction(2) ** e)
    return res


WIDE_RESULT_BYTES = 64 + 4 * L.RADIC_WIDE_LIMBS


def radic_det_exact_wide(A: torch.Tensor, options=None, out: Optional[torch.Tensor] = None,
                         workspace: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Enqueues the exact det_R(A) with up to RADIC_WIDE_MAX_PRIMES primes (radic_det_exact_wide);
    returns the device radic_wide_result buffer (not synchronised)."""
    _check_matrix(A)
    m, n = A.shape
    lib = L.lib()
    if out is None:
        out = torch.zeros(WIDE_RESULT_BYTES, dtype=torch.uint8, device=A.device)
    ws_bytes = int(lib.radic_wide_workspace_bytes(int(m), int(n), _opts(options)))
    if workspace is None:
        workspace = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=A.device)
    rc = lib.radic_det_exact_wide(A.data_ptr(), int(m), int(n), int(A.stride(0)), _TORCH_DTYPES[A.dtype],
                                  _opts(options), out.data_ptr(), workspace.data_ptr(), workspace.numel(),
                                  _stream(stream))
    L.check("radic_det_exact_wide", rc)
    return out


def parse_wide_result(buf: torch.Tensor) -> dict:
    """Host dictionary of a radic_wide_result buffer: the fields, the signed integer and the exact
    value as a Fraction (integer times 2^exact_exp)."""
    raw = buf.detach().to("cpu").contiguous().view(torch.uint8).numpy().tobytes()
    value, status, n_primes, exact_exp, sign, n_limbs, minors, _ = struct.unpack_from("<d7q", raw, 0)
    limbs = struct.unpack_from(f"<{L.RADIC_WIDE_LIMBS}I", raw, 64)
    mag = 0
    for i in reversed(range(L.RADIC_WIDE_LIMBS)):
        mag = (mag << 32) | limbs[i]
    integer = sign * mag
    return {"value": value, "status": status, "n_primes": n_primes, "exact_exp": exact_exp, "sign": sign,
            "n_limbs": n_limbs, "minors": minors, "integer": integer,
            "value_exact": Fraction(integer) * (Fraction(2) ** exact_exp)}


def det_exact_wide(A, options=None, stream=None) -> dict:
    """Convenience call of the wide exact mode: host (numpy) or device input, synchronises."""
    if isinstance(A, np.ndarray):
        A = torch.from_numpy(np.ascontiguousarray(A)).to("cuda")
    res = parse_wide_result(radic_det_exact_wide(A, options=options, stream=stream))
    if res["status"] != 0:
        raise L.RadicError("radic_det_exact_wide (device)", res["status"])
    return res


# ---------------------------------------------------------------------------
# Batches of matrices of uneven shape
# ---------------------------------------------------------------------------


TIERS = {"fp32": 1, "pair": 2}


def make_tuning(kind=None, task_cost=None, tol=0.0, growth_threshold=0.0, blocks_per_sm=0,
                prefix_depth=None, tiers=None, head_sharing=True, kernel_events=0) -> "L.RadicBatchTuning":
    """Batched-path tuning: `kind`, `task_cost` and `prefix_depth` map m to a mapping name, a task size
    and a prefix depth (2 or 3); `tiers` lists the low tiers the mixed router may use ("fp32",
    "pair"; default both; binary64 is always available); `head_sharing` factors each prefix head
    once for all its prefixes; `kernel_events` is the address of two cudaEvent_t recorded around
    the dominant kernel."""
    t = L.RadicBatchTuning()
    t.head_sharing = 0 if head_sharing else -1
    t.kernel_events = kernel_events or None
    if tiers is not None:
        mask = 0
        for name in tiers:
            mask |= TIERS[name]
        if mask == 0:
            raise ValueError("tiers must name at least one of " + ", ".join(TIERS))
        t.tiers = mask
    for m, d in (prefix_depth or {}).items():
        t.prefix_depth[int(m)] = int(d)
    for m, k in (kind or {}).items():
        t.kind[int(m)] = L.MAPPINGS[k] if isinstance(k, str) else int(k)
    for m, c in (task_cost or {}).items():
        t.task_cost[int(m)] = float(c)
    t.tol = tol
    t.growth_threshold = growth_threshold
    t.blocks_per_sm = blocks_per_sm
    return t


BATCH_TASK_KEYS = ["b", "tier", "kind", "shared", "group", "r0", "run", "lim", "vlo", "vhi"]


def batch_tasks_host(shapes, mode="mixed", tuning=None) -> list:
    """The tasks radic_batch_plan_create would make for these shapes, planned on the host only
    (radic_batch_plan_tasks_host): one dict per task with BATCH_TASK_KEYS, in task order."""
    shapes = [(int(m), int(n)) for m, n in shapes]
    batch = len(shapes)
    ms = (ctypes.c_int32 * batch)(*[m for m, _ in shapes])
    ns = (ctypes.c_int32 * batch)(*[n for _, n in shapes])
    offs, acc = [], 0
    for m, n in shapes:
        offs.append(acc)
        acc += m * n
    off = (ctypes.c_int64 * batch)(*offs)
    tun = ctypes.byref(tuning) if tuning is not None else None
    lib = L.lib()
    total = ctypes.c_int64(0)
    L.check("radic_batch_plan_tasks_host",
            lib.radic_batch_plan_tasks_host(ms, ns, off, batch, _mode(mode), tun, None, 0, ctypes.byref(total)))
    F = len(BATCH_TASK_KEYS)
    buf = (ctypes.c_int64 * (F * max(total.value, 1)))()
    L.check("radic_batch_plan_tasks_host",
            lib.radic_batch_plan_tasks_host(ms, ns, off, batch, _mode(mode), tun, buf, total.value, ctypes.byref(total)))
    return [dict(zip(BATCH_TASK_KEYS, [int(x) for x in buf[F * i:F * i + F]])) for i in range(total.value)]


class BatchPlan:
    """A plan for a batch of matrices (shapes and packing fixed), with its workspace.

    shapes: list of (m, n); matrix b is stored row-major (leading dimension n)
    at element offset offsets[b] of one packed device buffer.
    """

    def __init__(self, shapes, offsets=None, mode="mixed", tuning=None, device="cuda", stream=None):
        shapes = [(int(m), int(n)) for m, n in shapes]
        if offsets is None:
            offsets, acc = [], 0
            for m, n in shapes:
                offsets.append(acc)
                acc += m * n
        self.batch = len(shapes)
        self.shapes = shapes
        self.mode = mode
        self._m = (ctypes.c_int32 * self.batch)(*[m for m, _ in shapes])
        self._n = (ctypes.c_int32 * self.batch)(*[n for _, n in shapes])
        self._off = (ctypes.c_int64 * self.batch)(*[int(o) for o in offsets])
        self._tuning = tuning
        lib = L.lib()
        handle = ctypes.c_void_p()
        rc = lib.radic_batch_plan_create(self._m, self._n, self._off, self.batch, _mode(mode),
                                         ctypes.byref(tuning) if tuning is not None else None, ctypes.byref(handle))
        L.check("radic_batch_plan_create", rc)
        self._plan = handle
        self.ws_bytes = int(lib.radic_batch_workspace_bytes(self._plan))
        self.workspace = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=device)
        rc = lib.radic_batch_upload(self._plan, self.workspace.data_ptr(), self.workspace.numel(), _stream(stream))
        L.check("radic_batch_upload", rc)
        self._graphs = []

    INFO_KEYS = ["tasks_fp32", "tasks_fp64", "matrices_fp32", "matrices_fp64", "minors_fp32", "minors_fp64",
                 "blocks_fp32", "blocks_fp64", "tasks_pair", "matrices_pair", "minors_pair", "blocks_pair",
                 "launches", "dominant_m", "dominant_path", "dominant_tier"]

    def info(self) -> dict:
        buf = (ctypes.c_int64 * len(self.INFO_KEYS))()
        L.check("radic_batch_plan_info", L.lib().radic_batch_plan_info(self._plan, buf, len(self.INFO_KEYS)))
        return dict(zip(self.INFO_KEYS, [int(x) for x in buf]))

    def new_results(self) -> torch.Tensor:
        return torch.empty((self.batch, L.RESULT_WORDS), dtype=torch.int64, device=self.workspace.device)

    def radic_det_batched(self, A: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        if A.dtype not in _TORCH_DTYPES or not A.is_cuda:
            raise TypeError("A must be a packed CUDA tensor of a supported dtype")
        if out is None:
            out = self.new_results()
        rc = L.lib().radic_det_batched(self._plan, A.data_ptr(), _TORCH_DTYPES[A.dtype], out.data_ptr(),
                                       self.workspace.data_ptr(), self.workspace.numel(), _stream(stream))
        L.check("radic_det_batched", rc)
        return out

    def graph(self, A: torch.Tensor, out: torch.Tensor) -> "BatchGraph":
        g = BatchGraph(self, A, out)
        self._graphs.append(g)
        return g

    def close(self) -> None:
        for g in self._graphs:
            g.close()
        self._graphs = []
        if self._plan:
            L.lib().radic_batch_plan_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DetGraph:
    """A captured CUDA graph of one radic_det call on fixed buffers: replaying it runs the same
    kernels without the per-call planning and launch latency (radic_graph_create)."""

    def __init__(self, A: torch.Tensor, mode="fp64", options=None, out: Optional[torch.Tensor] = None,
                 workspace: Optional[torch.Tensor] = None):
        _check_matrix(A)
        m, n = A.shape
        md = _mode(mode)
        lib = L.lib()
        self.A = A
        self.out = out if out is not None else new_result(A.device)
        self._opts = L.make_options(**options) if isinstance(options, dict) else options
        ws_bytes = int(lib.radic_workspace_bytes(int(m), int(n), md, _opts(self._opts)))
        self.workspace = workspace if workspace is not None else torch.empty(max(ws_bytes, 256), dtype=torch.uint8,
                                                                             device=A.device)
        handle = ctypes.c_void_p()
        rc = lib.radic_graph_create(A.data_ptr(), int(m), int(n), int(A.stride(0)), _TORCH_DTYPES[A.dtype], md,
                                    _opts(self._opts), self.out.data_ptr(), self.workspace.data_ptr(),
                                    self.workspace.numel(), ctypes.byref(handle))
        L.check("radic_graph_create", rc)
        self._g = handle

    def launch(self, stream=None) -> None:
        L.check("radic_graph_launch", L.lib().radic_graph_launch(self._g, _stream(stream)))

    def close(self) -> None:
        if self._g:
            L.lib().radic_graph_destroy(self._g)
            self._g = None


class BatchGraph:
    """A captured CUDA graph of one batched call on fixed buffers."""

    def __init__(self, plan: BatchPlan, A: torch.Tensor, out: torch.Tensor):
        self.plan, self.A, self.out = plan, A, out  # keep the buffers alive
        handle = ctypes.c_void_p()
        rc = L.lib().radic_batch_graph_create(plan._plan, A.data_ptr(), _TORCH_DTYPES[A.dtype], out.data_ptr(),
                                              plan.workspace.data_ptr(), plan.workspace.numel(),
                                              ctypes.byref(handle))
        L.check("radic_batch_graph_create", rc)
        self._g = handle

    def launch(self, stream=None) -> None:
        L.check("radic_batch_graph_launch", L.lib().radic_batch_graph_launch(self._g, _stream(stream)))

    def close(self) -> None:
        if self._g:
            L.lib().radic_batch_graph_destroy(self._g)
            self._g = None


def parse_results(buf: torch.Tensor) -> list:
    """List of result dictionaries of a (batch, 16) result buffer."""
    host = buf.detach().to("cpu").contiguous()
    return [parse_result(host[b]) for b in range(host.shape[0])]
