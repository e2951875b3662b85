"""torch.autograd wrapper of the NURSD-1 forward: V = A(P, x).

Backward calls the library's gradient kernel (nursd_grad_points): given the
upstream gradient w = 2 dL/d conj(V) that autograd supplies for a real loss, it
returns A^H w for the phasors and Re sum_f P conj(d(A^H w)/dx) for the relay
positions.  The per-frequency fine grids are recomputed in backward, not
stored: forward saves only P and x.
"""
from __future__ import annotations

import torch


class _NursdForward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, P, xy, plan):
        plan.set_points(xy.detach().contiguous())
        V = plan.forward_phasor(P.detach().contiguous())
        ctx.plan = plan
        ctx.save_for_backward(P, xy)
        return V

    @staticmethod
    def backward(ctx, gV):
        P, xy = ctx.saved_tensors
        plan = ctx.plan
        plan.set_points(xy.detach().contiguous())  # another call may have moved the plan's samples
        gP, gxy = plan.grad_points(gV.detach().to(torch.complex64).contiguous(), P.detach().contiguous(),
                                   want_phasor=ctx.needs_input_grad[0], want_xy=ctx.needs_input_grad[1])
        return gP, gxy, None


def nursd_apply(plan, P: torch.Tensor, xy: torch.Tensor) -> torch.Tensor:
    """Differentiable NURSD-1 forward with `plan` (created with adjoint=True)."""
    return _NursdForward.apply(P, xy, plan)
