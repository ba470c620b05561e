"""The allocation-free entry point against the ordinary one.

radic_det_noalloc serves callers that cannot allocate device memory when
they need a determinant (their device memory belongs to another allocator or
a fixed pool, or their loop cannot take an allocation's synchronisation).  It
uses the library's static scratch array instead of a caller workspace.  This
file is collected last so that a run stopping at its first failure has already
run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1508_01326_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1508_01326_gb300 import build as B
    from paper_1508_01326_gb300 import _lib as L

    B.build()
    lib = L.lib()
    fn = lib.radic_det_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return lib


def _noalloc(lib, a, opts=None):
    import paper_1508_01326_gb300 as R

    out = R.new_result()
    rc = lib.radic_det_noalloc(a.data_ptr(), a.shape[0], a.shape[1], a.stride(0), 3,
                               ctypes.addressof(opts) if opts is not None else None, out.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    return rc, out


def _oracle(host):
    """Exact det_R and sum|terms| of a workload matrix from the oracle (stored values for 8 x 32)."""
    import oracle.radic_oracle as orc
    from tests.conftest import golden_abs_sums, golden_values

    if host.shape == (8, 32):
        return golden_values("fp64_8x32")[0], golden_abs_sums("fp64_8x32")[0]
    val, abs_sum = orc.radic_det_exact(host)
    return float(val), float(abs_sum)


def test_noalloc_matches_radic_det_on_two_calls_in_a_row(lib):
    import paper_1508_01326_gb300 as R
    from paper_1508_01326_gb300 import _lib as L

    mats = [W.uniform_matrix(41, 6, 20), W.fp64_8x32(), W.uniform_matrix(41, 6, 20)]
    for host in mats:
        want, scale = _oracle(host)
        a = torch.from_numpy(np.ascontiguousarray(host)).cuda()
        ref = R.parse_result(R.radic_det(a, mode="fp64"))
        rc, out = _noalloc(lib, a)
        assert rc == 0
        got = R.parse_result(out)
        assert got["status"] == 0 and got["minors"] == ref["minors"]
        # against the existing entry point, and against the oracle's exact value
        assert abs(got["value"] - ref["value"]) <= 1e-12 * scale
        assert abs(got["abs_sum"] - scale) <= 1e-12 * scale
        assert abs(got["value"] - want) <= 1e-12 * scale
        # with a fixed task schedule both entry points run the same kernels on
        # the same data: identical bits
        det_opts = L.make_options(deterministic=1)
        ref_fixed = R.parse_result(R.radic_det(a, mode="fp64", options=dict(deterministic=True)))
        rc, out = _noalloc(lib, a, det_opts)
        assert rc == 0
        fixed = R.parse_result(out)
        assert (fixed["value"], fixed["abs_sum"]) == (ref_fixed["value"], ref_fixed["abs_sum"])


def test_noalloc_rejects_plans_beyond_its_scratch(lib):
    from paper_1508_01326_gb300 import _lib as L

    a = torch.from_numpy(W.uniform_matrix(42, 6, 20)).cuda()
    opts = L.make_options(blocks=10000)  # 10000 partial slots need more than 128 KiB
    rc, _ = _noalloc(lib, a, opts)
    assert rc == 5  # RADIC_EWORKSPACE
