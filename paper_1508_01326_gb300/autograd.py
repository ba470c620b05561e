"""torch.autograd.Function for Radic's determinant of a batch of equal-shape matrices.

Forward: the batched path (prefix sharing), binary64 or the mixed router.
Backward: the hand-written kernel behind radic_det_backward_mode, which adds
each minor's signed cofactors sign(J) * det(M) * inv(M)^T into the gradient of
its columns (summed per prefix in closed form), with the eliminations in
binary64 or in pairs of binary32.
"""
from __future__ import annotations

import ctypes
from typing import Dict, Tuple

import torch

from . import _lib as L
from .api import BatchPlan, _stream

_PLANS: Dict[Tuple[int, int, int, int, str], BatchPlan] = {}


def _plan(batch: int, m: int, n: int, device: torch.device, mode: str = "fp64") -> BatchPlan:
    key = (batch, m, n, device.index if device.index is not None else torch.cuda.current_device(), mode)
    plan = _PLANS.get(key)
    if plan is None:
        plan = BatchPlan([(m, n)] * batch, [b * m * n for b in range(batch)], mode=mode, device=device)
        _PLANS[key] = plan
    return plan


def radic_det_backward(A: torch.Tensor, grad_out: torch.Tensor, stream=None, mode: str = "fp64") -> torch.Tensor:
    """Gradient of sum_b grad_out[b] * det_R(A[b]) with respect to A (batch, m, n); eliminations in
    binary64 (mode "fp64") or pairs of binary32 (mode "pair"), accumulation in binary64."""
    if A.dtype != torch.float64 or not A.is_cuda or A.dim() != 3:
        raise TypeError("A must be a (batch, m, n) float64 CUDA tensor")
    A = A.contiguous()
    batch, m, n = A.shape
    grad_out = grad_out.to(dtype=torch.float64, device=A.device).contiguous()
    grad = torch.empty_like(A)
    lib = L.lib()
    ws_bytes = int(lib.radic_backward_workspace_bytes(batch, m, n))
    ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=A.device)
    rc = lib.radic_det_backward_mode(A.data_ptr(), batch, m, n, n, m * n, grad_out.data_ptr(), grad.data_ptr(),
                                     ws.data_ptr(), ws.numel(), L.MODES[mode], _stream(stream))
    L.check("radic_det_backward_mode", rc)
    return grad


class RadicDet(torch.autograd.Function):
    """det_R of each matrix of a (batch, m, n) float64 CUDA tensor, differentiable.

    precision "fp64": binary64 forward and backward; "mixed": the batched mixed router forward
    (pairs of binary32 where they meet its 1e-10 target) and the pair backward."""

    @staticmethod
    def forward(ctx, A: torch.Tensor, precision: str = "fp64") -> torch.Tensor:
        if A.dtype != torch.float64 or not A.is_cuda or A.dim() != 3:
            raise TypeError("A must be a (batch, m, n) float64 CUDA tensor")
        if precision not in ("fp64", "mixed"):
            raise ValueError("precision must be 'fp64' or 'mixed'")
        A = A.contiguous()
        batch, m, n = A.shape
        plan = _plan(batch, m, n, A.device, precision)
        out = plan.radic_det_batched(A.reshape(-1))
        ctx.save_for_backward(A)
        ctx.precision = precision
        return out.view(torch.float64)[:, 0].clone()

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (A,) = ctx.saved_tensors
        mode = "pair" if ctx.precision == "mixed" else "fp64"
        return radic_det_backward(A, grad_out, mode=mode), None


def radic_det_autograd(A: torch.Tensor, precision: str = "fp64") -> torch.Tensor:
    """Differentiable det_R: (m, n) -> scalar, (batch, m, n) -> (batch,)."""
    if A.dim() == 2:
        return RadicDet.apply(A.unsqueeze(0), precision)[0]
    return RadicDet.apply(A, precision)
