"""Radic's determinant of non-square matrices on NVIDIA GB300 (sm_103a).

det_R(A) = sum over ascending column sequences J of (-1)^(r+s) det(A[:, J])
(Definition 3, Eq. (1) of arXiv 1508.01326), computed by hand-written CUDA
kernels in the in-tree shared library libradic.so behind the C ABI of
include/radic.h.  This package is the thin Python binding; the shared
library is loaded on first use and its absence is an error.
"""
from ._lib import RadicError, make_options  # noqa: F401
from .autograd import RadicDet, radic_det_autograd, radic_det_backward  # noqa: F401
from .api import (  # noqa: F401
    BatchGraph,
    BatchPlan,
    DetGraph,
    det,
    det_exact_wide,
    make_tuning,
    parse_results,
    new_result,
    parse_result,
    parse_wide_result,
    radic_det,
    radic_det_exact_wide,
    radic_plan_info,
    prefix_plan_host,
    batch_tasks_host,
    radic_primes,
    radic_status_string,
    radic_terms,
    radic_unrank,
    radic_version,
    radic_workspace_bytes,
)
