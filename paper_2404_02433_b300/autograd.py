"""kappa_eff as a differentiable function of the voxel log-conductivity.

``effective_conductivity(log_kappa, direction)`` returns the ETC of
Eq. (effective formula dis) as a 0-d tensor.  When log_kappa requires a
gradient, the forward call runs the library's adjoint together with the solve
(etc_gradient: one extra PCG solve and one gradient kernel) and the backward
pass only scales the stored gradient; otherwise (torch.no_grad, or a tensor
without requires_grad) it runs the forward solve alone.  The exponential that
maps log_kappa to kappa is the only torch computation.
"""
from __future__ import annotations

import torch

from . import binding as B


def _check_input(log_kappa):
    if log_kappa.dtype != torch.float64 or not log_kappa.is_cuda or log_kappa.dim() != 3:
        raise ValueError("log_kappa must be a 3-D float64 CUDA tensor (nz, ny, nx)")


def _solve_only(log_kappa, direction, lengths, rtol, p_in, p_out):
    _check_input(log_kappa)
    rve = B.RVE(torch.exp(log_kappa).contiguous(), lengths=lengths)
    try:
        k, info = rve.solve(direction, p_in=p_in, p_out=p_out, rtol=rtol)
    finally:
        rve.close()
    if info["status"] != B.ETC_OK:
        raise B.EtcError(info["status"], "the forward solve did not converge")
    return torch.tensor(k, dtype=torch.float64, device=log_kappa.device)


class EffectiveConductivity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_kappa, direction, lengths, rtol, p_in, p_out):
        _check_input(log_kappa)
        rve = B.RVE(torch.exp(log_kappa).contiguous(), lengths=lengths)
        try:
            grad, k, _ = rve.gradient(direction, p_in=p_in, p_out=p_out, rtol=rtol)
        finally:
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
    if torch.is_grad_enabled() and log_kappa.requires_grad:
        return EffectiveConductivity.apply(log_kappa, direction, tuple(lengths), rtol, p_in, p_out)
    return _solve_only(log_kappa, direction, tuple(lengths), rtol, p_in, p_out)
