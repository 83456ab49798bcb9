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
The backward pass is a fresh solve: nothing of the forward Krylov bases is stored (only Z,
for dL/dt), so memory is that of one forward call.
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


def transpose_plan(plan: Plan, **kw) -> Plan:
    """A plan for A^T (same grid and diffusion, velocity negated), same options."""
    opts = dict(p_max=plan.p_max, m=plan.m, tol=plan.tol, max_cycles=plan.max_cycles,
                algorithm=plan.algorithm, precision=plan.precision)
    opts.update(kw)
    return Plan(plan.sides, plan.diff, tuple(-v for v in plan.vel), stream=plan.stream, **opts)


class _ExpmBlock(torch.autograd.Function):
    @staticmethod
    def forward(ctx, t, B, plan, plan_T):
        tt = float(t)
        Z, info = plan.expm_block(tt, _as_colmajor(B.detach()))
        ctx.save_for_backward(Z)
        ctx.plan, ctx.plan_T, ctx.t = plan, plan_T, tt
        return Z

    @staticmethod
    def backward(ctx, G):
        (Z,) = ctx.saved_tensors
        G = _as_colmajor(G.detach())
        dB = dt = None
        if ctx.needs_input_grad[1]:
            dB, _ = ctx.plan_T.expm_block(ctx.t, G)
        if ctx.needs_input_grad[0]:
            AZ = ctx.plan.op_apply(1.0, Z)                # A Z (t folded out)
            dt = (G * AZ).sum().reshape(())
        return dt, dB, None, None


def expm_block(t, B, plan: Plan, plan_T: Plan | None = None):
    """Differentiable Z = r(tA) B.  t: 0-d float64 tensor (may require grad), B: (n, p)
    float64 CUDA tensor (may require grad).  plan_T defaults to transpose_plan(plan)."""
    if plan_T is None:
        plan_T = transpose_plan(plan)
    if not torch.is_tensor(t):
        t = torch.tensor(float(t), dtype=torch.float64, device=B.device)
    return _ExpmBlock.apply(t, B, plan, plan_T)
