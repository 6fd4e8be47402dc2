"""torch.autograd.Function around the checkpointed forward/adjoint sweep.

`final_energy(u0, solver, horizon)` returns E(tau0 + horizon) (Eq. 2.1) of the
perturbation started from the device field u0 (complex128, layout of
include/pnop.h).  Its forward half runs the checkpointed forward sweep in the
C library (binomial checkpoints, Section 2.5, Eq. 2.18-2.20; with
snap_budget <= 0 the pool is sized to the context's HBM budget); its backward
is the library's hand-written adjoint sweep (the exact transpose of the
discrete step), entered with the incoming cotangent of E.  The gradient
returned to autograd is the Euclidean one of the stored real and imaginary
parts, d/dRe + i d/dIm, which is PyTorch's convention for a real loss of a
complex tensor.  u0 is used as given (no rescaling to an energy shell), so E
is a plain function of u0.

One forward may be pending per context: calling other context entry points
between forward and backward discards the sweep and the backward raises.
"""
from __future__ import annotations

import torch

from . import _lib


class FinalEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0: torch.Tensor, solver: "_lib.Context", horizon: float):
        if u0.dtype != torch.complex128 or not u0.is_cuda or tuple(u0.shape) != tuple(solver.shape):
            raise ValueError("u0 must be a complex128 CUDA tensor of shape %s" % (solver.shape,))
        x = u0.detach().contiguous()
        ET, _ = solver.pnop_gradient_forward(x, -1.0, horizon)
        ctx.solver = solver
        ctx.meta = (u0.shape, u0.device)
        return torch.tensor(ET, dtype=torch.float64, device=u0.device)

    @staticmethod
    def backward(ctx, gE: torch.Tensor):
        shape, device = ctx.meta
        g = torch.empty(shape, dtype=torch.complex128, device=device)
        ctx.solver.pnop_gradient_backward(float(gE.item()), g, euclidean=True)
        return g, None, None


def final_energy(u0: torch.Tensor, solver: "_lib.Context", horizon: float) -> torch.Tensor:
    """E(tau0 + horizon) as a differentiable function of the device field u0."""
    return FinalEnergy.apply(u0, solver, horizon)
