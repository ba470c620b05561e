"""ctypes declarations of the C ABI in include/radic.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libradic.so")

RADIC_MAX_M = 32
RADIC_MAX_N = 64
RADIC_MAX_PRIMES = 4
RADIC_WIDE_MAX_PRIMES = 32
RADIC_WIDE_LIMBS = 32

STATUS = {0: "RADIC_OK", 1: "RADIC_EINVAL", 2: "RADIC_EOVERFLOW", 3: "RADIC_ECUDA", 4: "RADIC_ETIMEOUT",
          5: "RADIC_EWORKSPACE", 6: "RADIC_EUNSUPPORTED"}
DTYPES = {"int8": 0, "int32": 1, "float32": 2, "float64": 3}
MODES = {"fp64": 0, "mixed": 1, "exact": 2, "pair": 3}
MAPPINGS = {"auto": 0, "thread": 1, "group": 2, "prefix": 3}


class RadicOptions(ctypes.Structure):
    _fields_ = [
        ("mapping", ctypes.c_int32),
        ("group_width", ctypes.c_int32),
        ("ranks_per_task", ctypes.c_int32),
        ("threads_per_block", ctypes.c_int32),
        ("blocks", ctypes.c_int32),
        ("flag_capacity", ctypes.c_int32),
        ("growth_threshold", ctypes.c_double),
        ("kernel_events", ctypes.c_void_p),
        ("prefix_depth", ctypes.c_int32),
        ("lanes_per_prefix", ctypes.c_int32),
        ("deterministic", ctypes.c_int32),
        ("reserved32", ctypes.c_int32),
        ("reserved", ctypes.c_int64 * 1),
    ]


RESULT_WORDS = 16  # radic_result is sixteen 8-byte words


class RadicBatchTuning(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32 * (RADIC_MAX_M + 1)),
        ("task_cost", ctypes.c_double * (RADIC_MAX_M + 1)),
        ("tol", ctypes.c_double),
        ("growth_threshold", ctypes.c_double),
        ("blocks_per_sm", ctypes.c_int32),
        ("prefix_depth", ctypes.c_int32 * (RADIC_MAX_M + 1)),
        ("tiers", ctypes.c_int32),
        ("head_sharing", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 5),
        ("kernel_events", ctypes.c_void_p),
    ]

_lib = None


class RadicError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed: {STATUS.get(code, code)}")
        self.code = code


def lib() -> ctypes.CDLL:
    """The loaded libradic.so.  Raises if the library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it with paper_1508_01326_gb300.build.build() "
            "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, sz, i32, i64, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
    opt = ctypes.POINTER(RadicOptions)
    L.radic_status_string.argtypes = [i32]
    L.radic_status_string.restype = ctypes.c_char_p
    L.radic_version.argtypes = []
    L.radic_version.restype = i32
    L.radic_primes.argtypes = [ctypes.POINTER(ctypes.c_uint32), i32]
    L.radic_primes.restype = i32
    L.radic_workspace_bytes.argtypes = [i32, i32, i32, opt]
    L.radic_workspace_bytes.restype = sz
    L.radic_det.argtypes = [vp, i32, i32, i64, i32, i32, opt, vp, vp, sz, vp]
    L.radic_det.restype = i32
    L.radic_terms.argtypes = [vp, i32, i32, i64, i32, i32, opt, u64, u64, vp, vp]
    L.radic_terms.restype = i32
    L.radic_unrank.argtypes = [i32, i32, u64, u64, vp, opt, vp]
    L.radic_unrank.restype = i32
    _declare_optional(L)
    _lib = L
    return L


def _declare_optional(L: ctypes.CDLL) -> None:
    """Declarations of the batched, backward and allocation-free entry points."""
    vp, sz, i32, i64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int64
    pp = ctypes.POINTER(vp)
    table = {
        "radic_batch_plan_create": ([vp, vp, vp, i32, i32, vp, pp], i32),
        "radic_batch_plan_destroy": ([vp], i32),
        "radic_batch_plan_info": ([vp, ctypes.POINTER(i64), i32], i32),
        "radic_plan_info": ([i32, i32, i32, ctypes.POINTER(RadicOptions), ctypes.POINTER(i64), i32], i32),
        "radic_prefix_plan_host": ([i32, i32, i32, ctypes.POINTER(RadicOptions), i32, i32, ctypes.POINTER(i64), i32],
                                   i32),
        "radic_batch_plan_tasks_host": ([vp, vp, vp, i32, i32, vp, ctypes.POINTER(i64), i64, ctypes.POINTER(i64)], i32),
        "radic_batch_workspace_bytes": ([vp], sz),
        "radic_batch_upload": ([vp, vp, sz, vp], i32),
        "radic_det_batched": ([vp, vp, i32, vp, vp, sz, vp], i32),
        "radic_graph_create": ([vp, i32, i32, i64, i32, i32, ctypes.POINTER(RadicOptions), vp, vp, sz, pp], i32),
        "radic_graph_launch": ([vp, vp], i32),
        "radic_graph_destroy": ([vp], i32),
        "radic_batch_graph_create": ([vp, vp, i32, vp, vp, sz, pp], i32),
        "radic_batch_graph_launch": ([vp, vp], i32),
        "radic_batch_graph_destroy": ([vp], i32),
        "radic_backward_workspace_bytes": ([i32, i32, i32], sz),
        "radic_det_backward": ([vp, i32, i32, i32, i64, i64, vp, vp, vp, sz, vp], i32),
        "radic_det_backward_mode": ([vp, i32, i32, i32, i64, i64, vp, vp, vp, sz, i32, vp], i32),
        "radic_det_noalloc": ([vp, i32, i32, i64, i32, vp, vp, vp], i32),
        "radic_wide_workspace_bytes": ([i32, i32, ctypes.POINTER(RadicOptions)], sz),
        "radic_det_exact_wide": ([vp, i32, i32, i64, i32, ctypes.POINTER(RadicOptions), vp, vp, sz, vp], i32),
    }
    for name, (args, res) in table.items():
        fn = getattr(L, name, None)
        if fn is not None:
            fn.argtypes = args
            fn.restype = res


def check(fn: str, code: int) -> None:
    if code != 0:
        raise RadicError(fn, code)


def make_options(mapping: str | int = 0, group_width: int = 0, ranks_per_task: int = 0,
                 threads_per_block: int = 0, blocks: int = 0, flag_capacity: int = 0,
                 growth_threshold: float = 0.0, kernel_events: int = 0, prefix_depth: int = 0,
                 lanes_per_prefix: int = 0, deterministic: bool = False) -> RadicOptions:
    o = RadicOptions()
    o.mapping = MAPPINGS[mapping] if isinstance(mapping, str) else int(mapping)
    o.group_width = group_width
    o.ranks_per_task = ranks_per_task
    o.threads_per_block = threads_per_block
    o.blocks = blocks
    o.flag_capacity = flag_capacity
    o.growth_threshold = growth_threshold
    o.kernel_events = kernel_events or None
    o.prefix_depth = prefix_depth
    o.lanes_per_prefix = lanes_per_prefix
    o.deterministic = 1 if deterministic else 0
    return o
