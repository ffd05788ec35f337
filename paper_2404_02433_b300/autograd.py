"""kappa_eff as a differentiable function of the voxel log-conductivity.

``effective_conductivity(log_kappa, direction)`` returns the ETC of
Eq. (effective formula dis) as a 0-d tensor; its backward pass runs the
library's adjoint (one extra PCG solve and one gradient kernel, etc_gradient).
The exponential that maps log_kappa to kappa is the only torch computation.
"""
from __future__ import annotations

import torch

from . import binding as B


class EffectiveConductivity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_kappa, direction, lengths, rtol, p_in, p_out):
        if log_kappa.dtype != torch.float64 or not log_kappa.is_cuda or log_kappa.dim() != 3:
            raise ValueError("log_kappa must be a 3-D float64 CUDA tensor (nz, ny, nx)")
        kappa = torch.exp(log_kappa).contiguous()
        rve = B.RVE(kappa, lengths=lengths)
        grad, k, _ = rve.gradient(direction, p_in=p_in, p_out=p_out, rtol=rtol)
        rve.close()
        ctx.save_for_backward(grad)
        return torch.tensor(k, dtype=torch.float64, device=log_kappa.device)

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return grad_out * grad, None, None, None, None, None


def effective_conductivity(log_kappa, direction=2, lengths=(1.0, 1.0, 1.0), rtol=1e-10,
                           p_in=1.0, p_out=0.0):
    """kappa_eff of an isotropic medium kappa = exp(log_kappa), differentiable."""
    return EffectiveConductivity.apply(log_kappa, direction, tuple(lengths), rtol, p_in, p_out)
