"""GPU parity of the hand-written backward kernel.

The gradient of det_R is checked against the oracle's exact gradient
(d det_R / d a_ij = (-1)^(i+j) det_R(A without row i and column j), enumerated
on small cases, Pfaffian closed form on the 6 x 28 workload), against central
finite differences with h = 1e-6 (exact up to rounding, since det_R is affine in
every entry), and with torch.autograd.gradcheck.
"""
import numpy as np
import pytest
import torch

import oracle.radic_oracle as orc
from paper_1508_01326_gb300 import workloads as W
from tests.conftest import golden_abs_sums

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1508_01326_gb300 import build as B

    B.build()


def R():
    import paper_1508_01326_gb300 as R_

    return R_


@pytest.mark.parametrize("mode", ["fp64", "pair"])
@pytest.mark.parametrize("m,n", [(1, 6), (2, 5), (3, 7), (4, 9), (5, 5), (6, 10), (7, 10), (8, 11), (4, 3),
                                 (3, 14), (5, 16), (8, 13)])
def test_backward_matches_exact_gradient(m, n, mode):
    rng = np.random.default_rng(100 * m + n)
    mats = rng.uniform(-1, 1, (3, m, n))
    A = torch.from_numpy(mats).cuda()
    g_out = torch.tensor([1.0, -2.5, 0.75], dtype=torch.float64, device="cuda")
    grad = R().radic_det_backward(A, g_out, mode=mode).cpu().numpy()
    for b in range(3):
        if m > n:
            want = np.zeros((m, n))
        else:
            want = np.array([[float(x) for x in row] for row in orc.radic_grad_exact(mats[b], use_pfaffian=False)])
        scale = max(np.abs(want).max(), 1e-300)
        assert np.abs(grad[b] - float(g_out[b]) * want).max() <= 1e-11 * scale * max(1.0, abs(float(g_out[b])))


@pytest.mark.parametrize("mode", ["fp64", "pair"])
def test_backward_singular_prefixes(mode):
    # integer entries with a repeated column and a zero column: prefixes that
    # contain both copies, or the zero column, have an exactly zero pivot and
    # take the per-minor path for their leaves
    a = W.integer_matrix(17, 5, 10, 4, np.int32).astype(np.float64)
    a[:, 3] = a[:, 1]
    a[:, 6] = 0.0
    mats = np.stack([a, W.integer_matrix(18, 5, 10, 4, np.int32).astype(np.float64)])
    grad = R().radic_det_backward(torch.from_numpy(mats).cuda(), torch.ones(2, dtype=torch.float64, device="cuda"),
                                  mode=mode).cpu().numpy()
    for b in range(2):
        want = np.array([[float(x) for x in row] for row in orc.radic_grad_exact(mats[b], use_pfaffian=False)])
        assert np.abs(grad[b] - want).max() <= 1e-11 * max(np.abs(want).max(), 1.0)


def test_autograd_function_and_gradcheck():
    A = torch.from_numpy(W.uniform_matrix(5, 3, 6)).cuda().unsqueeze(0).requires_grad_(True)
    # the prefix backward adds in a fixed order except on its singular-prefix
    # path, which (like the per-minor backward for m <= 2) uses shared-memory
    # atomics; nondet_tol covers that addition order
    assert torch.autograd.gradcheck(R().RadicDet.apply, (A,), eps=1e-6, atol=1e-7, rtol=1e-6, nondet_tol=1e-12)
    x = torch.from_numpy(W.uniform_matrix(6, 4, 8)).cuda().requires_grad_(True)
    y = R().radic_det_autograd(x)
    y.backward()
    want = np.array([[float(v) for v in row] for row in orc.radic_grad_exact(x.detach().cpu().numpy(),
                                                                               use_pfaffian=False)])
    assert np.abs(x.grad.cpu().numpy() - want).max() <= 1e-11 * np.abs(want).max()


# sum|terms| of each 6 x 28 matrix from the oracle's binary64 host enumeration
# (tests/golden/workload_abs_sum.txt): the tolerance scale of the forward values
ABS = golden_abs_sums("diff_256x6x28")


@pytest.fixture(scope="module")
def diff_batch():
    return W.diff_256x6x28()


def test_full_diff_256x6x28_forward_and_backward(diff_batch):
    A = torch.from_numpy(diff_batch).cuda().requires_grad_(True)
    vals = R().radic_det_autograd(A)
    vals.sum().backward()
    grad = A.grad.cpu().numpy()
    # forward against the Pfaffian closed form on a few matrices
    for b in (0, 97, 255):
        exact = orc.radic_det_pfaffian(diff_batch[b])
        assert abs(float(vals[b].detach()) - float(exact)) <= 1e-12 * ABS[b]
    # backward against the exact adjugate gradient (Pfaffian form) for matrix 0
    want = np.array([[float(v) for v in row] for row in orc.radic_grad_exact(diff_batch[0], use_pfaffian=True)])
    assert np.abs(grad[0] - want).max() <= 1e-10 * np.abs(want).max()
    # central finite differences (h = 1e-6) through the GPU forward on sampled entries
    rng = np.random.default_rng(0)
    base = torch.from_numpy(diff_batch.copy()).cuda()
    h = 1e-6
    for _ in range(12):
        b, i, j = int(rng.integers(256)), int(rng.integers(6)), int(rng.integers(28))
        plus = base.clone()
        minus = base.clone()
        plus[b, i, j] += h
        minus[b, i, j] -= h
        fd = (float(R().radic_det_autograd(plus)[b]) - float(R().radic_det_autograd(minus)[b])) / (2 * h)
        assert abs(fd - grad[b, i, j]) <= 1e-6 * max(1.0, np.abs(grad[b]).max())


def test_full_diff_256x6x28_mixed_precision(diff_batch):
    # mixed forward (pairs of binary32 at the 1e-10 target) and pair backward
    A = torch.from_numpy(diff_batch).cuda().requires_grad_(True)
    vals = R().radic_det_autograd(A, precision="mixed")
    vals.sum().backward()
    grad = A.grad.cpu().numpy()
    for b in (0, 128):
        exact = orc.radic_det_pfaffian(diff_batch[b])
        assert abs(float(vals[b].detach()) - float(exact)) <= 1e-10 * ABS[b]
    want = np.array([[float(v) for v in row] for row in orc.radic_grad_exact(diff_batch[0], use_pfaffian=True)])
    assert np.abs(grad[0] - want).max() <= 1e-10 * np.abs(want).max()


@pytest.mark.parametrize("mode", ["fp64", "pair"])
def test_backward_prefix_deterministic(diff_batch, mode):
    # with no singular prefix the prefix backward adds every entry in a fixed
    # order (per-warp tiles, no atomics): repeated calls agree bit for bit
    A = torch.from_numpy(diff_batch[:64]).cuda()
    g = torch.ones(64, dtype=torch.float64, device="cuda")
    first = R().radic_det_backward(A, g, mode=mode)
    for _ in range(3):
        assert torch.equal(R().radic_det_backward(A, g, mode=mode), first)


def _column_norm_symmetric_sum(a):
    # e_m of the column norms: by Hadamard's inequality an upper bound of
    # sum over J of |det A[:, J]|, computed on the host without the GPU
    m = a.shape[0]
    e = np.zeros(m + 1)
    e[0] = 1.0
    for x in np.linalg.norm(a, axis=0):
        for k in range(m, 0, -1):
            e[k] += x * e[k - 1]
    return e[m]


@pytest.mark.parametrize("mode,tol", [("fp64", 1e-12), ("pair", 1e-10)])
@pytest.mark.parametrize("m,n", [(3, 64), (4, 40), (6, 24), (8, 20)])
def test_backward_long_rows_against_central_differences(m, n, mode, tol):
    # many candidate columns per prefix (the largest column buffers and
    # tiles); det_R is affine in every entry, so the central difference with
    # step 1 through the oracle's binary64 enumeration is the gradient entry
    # up to rounding
    from oracle import cpu_enum

    rng = np.random.default_rng(1000 * m + n)
    a = rng.uniform(-1, 1, (m, n))
    grad = R().radic_det_backward(torch.from_numpy(a[None].copy()).cuda(),
                                  torch.ones(1, dtype=torch.float64, device="cuda"), mode=mode).cpu().numpy()[0]
    scale = 0.0
    for i in range(m):
        for j in range(n):
            p, q = a.copy(), a.copy()
            p[i, j] += 1.0
            q[i, j] -= 1.0
            fp, sp, _ = cpu_enum.radic_cpu_sum(p)
            fq, sq, _ = cpu_enum.radic_cpu_sum(q)
            scale = max(scale, sp, sq)
            assert abs(grad[i, j] - (fp - fq) / 2) <= tol * scale, (i, j, grad[i, j], (fp - fq) / 2)


@pytest.mark.parametrize("mode,tol", [("fp64", 1e-12), ("pair", 1e-10)])
def test_backward_largest_tiles_row_identity(mode, tol):
    # m = 8, n = 64: the largest shared-memory layout.  det_R is linear in
    # each row, so sum_j a_ij d det_R / d a_ij = det_R(A) for every row i
    # (Euler's identity, the Laplace expansion of every minor along row i),
    # checked against the binary64 forward value
    a = W.uniform_matrix(41, 8, 64)
    grad = R().radic_det_backward(torch.from_numpy(a[None].copy()).cuda(),
                                  torch.ones(1, dtype=torch.float64, device="cuda"), mode=mode).cpu().numpy()[0]
    det = R().det(a, mode="fp64")["value"]
    bound = _column_norm_symmetric_sum(a)
    for i in range(8):
        assert abs(float(np.dot(a[i], grad[i])) - det) <= tol * bound, (i, float(np.dot(a[i], grad[i])), det)
