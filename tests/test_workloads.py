"""The seeded workloads match their stated recipes (shapes, types, ranges, minor
counts), so that tests, bench and oracle draw the same inputs (no GPU)."""
import math

import numpy as np

from paper_1508_01326_gb300 import workloads as W


def test_single_matrix_workloads():
    a = W.int_3x12()
    assert a.shape == (3, 12) and a.dtype == np.int32 and a.min() >= -9 and a.max() <= 9
    x = W.fp64_8x32()
    assert x.shape == (8, 32) and x.dtype == np.float64 and x.min() >= -1.0 and x.max() < 1.0
    assert math.comb(32, 8) == 10518300
    e = W.int8_12x40()
    assert e.shape == (12, 40) and e.dtype == np.int8 and e.min() >= -3 and e.max() <= 3
    assert np.array_equal(W.int8_10x24(), e[:10, :24])
    assert math.comb(40, 12) == 5586853480 and math.comb(24, 10) == 1961256
    d = W.diff_256x6x28()
    assert d.shape == (256, 6, 28) and d.min() >= -1.0 and d.max() < 1.0
    assert 256 * math.comb(28, 6) == 96445440
    # reproducible draws
    assert np.array_equal(W.fp64_8x32(), x) and np.array_equal(W.int_3x12(), a)


def test_batched_workload():
    mats = W.batched_4096()
    assert len(mats) == 4096
    ms = np.array([a.shape[0] for a in mats])
    ds = np.array([a.shape[1] - a.shape[0] for a in mats])
    assert ms.min() == 2 and ms.max() == 10 and ds.min() == 1 and ds.max() == 20
    assert sum(math.comb(a.shape[1], a.shape[0]) for a in mats) == 3373693081
    # N(0,1) entries: sample moments near 0 and 1
    flat = np.concatenate([a.ravel() for a in mats])
    assert abs(flat.mean()) < 0.01 and abs(flat.std() - 1.0) < 0.01


def test_pack_batch_layout():
    mats = [W.uniform_matrix(1, 2, 5), W.uniform_matrix(2, 3, 4), W.uniform_matrix(3, 1, 7)]
    data, ms, ns, offs = W.pack_batch(mats, np.float32)
    assert data.dtype == np.float32 and list(ms) == [2, 3, 1] and list(ns) == [5, 4, 7]
    assert list(offs) == [0, 10, 22] and data.size == 29
    for a, o in zip(mats, offs):
        m, n = a.shape
        assert np.array_equal(data[o:o + m * n].reshape(m, n), a.astype(np.float32))
