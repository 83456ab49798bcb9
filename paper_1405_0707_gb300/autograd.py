"""Differentiation of Z = r(tA) B: a hand-written adjoint behind torch.autograd.Function.

For a loss L(Z) with G = dL/dZ:
  dL/dB = r(tA)^T G = r(tA^T) G      (r has real coefficients, so r(M)^T = r(M^T)); computed
                                      by the same shifted block FOM on A^T.  For the
                                      convection-diffusion family, A^T is the same stencil
                                      with the velocity negated (central differences:
                                      (v . grad_h)^T = -v . grad_h).
  dL/dt = <G, A Z>                    d/dt e^{tA} B = A e^{tA} B; this is the derivative of
                                      the exponential that r approximates (it differs from
                                      the derivative of r(tA) B by the CF error of r').
The backward pass is one call of the library's expm_block_adjoint: a fresh solve with A^T
(nothing of the forward Krylov bases is stored, only Z for dL/dt, so memory is that of one
forward call plus the companion plan of A^T) and the inner product on the device.
"""
from __future__ import annotations

import torch

from .api import Plan, colmajor


def _as_colmajor(X):
    if X.dim() == 2 and (X.stride(0) == 1 or X.shape[1] == 1) and X.dtype == torch.float64:
        return X
    Y = colmajor(X.shape[0], X.shape[1], device=X.device)
    Y.copy_(X)
    return Y


class _ExpmBlock(torch.autograd.Function):
    @staticmethod
    def forward(ctx, t, B, plan):
        tt = float(t)
        Z, info = plan.expm_block(tt, _as_colmajor(B.detach()))
        ctx.save_for_backward(Z)
        ctx.plan, ctx.t = plan, tt
        return Z

    @staticmethod
    def backward(ctx, G):
        (Z,) = ctx.saved_tensors
        G = _as_colmajor(G.detach())
        want_dB, want_dt = bool(ctx.needs_input_grad[1]), bool(ctx.needs_input_grad[0])
        if not (want_dB or want_dt):
            return None, None, None
        dB, gt, _ = ctx.plan.expm_block_adjoint(ctx.t, G, Z, want_dB=want_dB, want_dt=want_dt)
        dt = torch.tensor(gt, dtype=torch.float64, device=G.device) if want_dt else None
        return dt, dB, None


def expm_block(t, B, plan: Plan):
    """Differentiable Z = r(tA) B.  t: 0-d float64 tensor (may require grad), B: (n, p)
    float64 CUDA tensor (may require grad).  The backward pass is one library call
    (expm_block_adjoint): dL/dB by the method on A^T, dL/dt = <G, A Z> on the device."""
    if not torch.is_tensor(t):
        t = torch.tensor(float(t), dtype=torch.float64, device=B.device)
    return _ExpmBlock.apply(t, B, plan)
