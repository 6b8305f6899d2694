"""Demag energy as a differentiable function of m (torch.autograd.Function).

Forward calls ``demag_energy`` (phi = P m, h_d = -D phi, E = -1/2 V sum m.h_d,
all in CUDA kernels) and, when m requires grad, the same call also returns
dE/dm = 1/2 V (D P m + P^T D^T m) from the hand-written adjoint; backward
scales that saved gradient by the incoming grad.  With precision "fft_field"
the energy of the analytic collocation field is used instead
(``demag_energy_field_fft``: one 3D FFT convolution, dE/dm = -V h_d).
"""
from __future__ import annotations

import torch

from . import _abi


class DemagEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, plan, precision="fp32"):
        if m.dtype != torch.float32 or not m.is_cuda:
            raise ValueError("m must be a float32 CUDA tensor [3][n3][n2][n1]")
        m = m.contiguous()
        e = torch.empty((), dtype=torch.float64, device=m.device)
        grad = torch.empty_like(m) if ctx.needs_input_grad[0] else None
        if precision == "fft_field":
            _abi.demag_energy_field_fft(plan, m, e, grad)
        else:
            _abi.demag_energy(plan, m, e, grad, precision)
        ctx.save_for_backward(grad if grad is not None else torch.empty(0, device=m.device))
        return e

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        return (gout.to(grad.dtype) * grad, None, None)


def demag_energy_fn(m: torch.Tensor, plan, precision: str = "fp32") -> torch.Tensor:
    """Energy E(m) (0-dim float64 tensor) with autograd support."""
    return DemagEnergy.apply(m, plan, precision)
