"""Differentiable trap fields: a torch.autograd.Function over the engine's kernels.

V = trap_fields(holo, phi) evaluates Eq. 1 (V_m = (1/N) sum_j exp(i (phi_j - Delta_j^m)))
for float32 CUDA phases phi with the traps of `holo` (a hot.Hologram), and its backward
pass runs the adjoint kernel, dL/dphi_j = (1/N) Im[exp(-i phi_j) sum_m G_m exp(i Delta_j^m)]
with G = the incoming complex gradient (PyTorch's convention, 2 dL/d conj V).  Both run
on the Hologram's CUDA stream, which should be the stream autograd runs on (the current
stream when the Hologram was created).

trap_intensity_loss implements the loss of the differentiable configuration,
L = -sum_m log |V_m|^2 + beta * var_m |V_m|^2 (population variance).

intensity_loss(holo, phi, beta) is the same loss as one library call (hot_intensity_loss: the
forward field, the loss and its adjoint coefficients, and the adjoint, all on the device), with
the gradient kept for backward: an optimiser step then costs three kernels and the update.
"""
from __future__ import annotations

import torch

from . import hot


class TrapFields(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi: torch.Tensor, holo: "hot.Hologram") -> torch.Tensor:
        assert phi.is_cuda and phi.dtype == torch.float32 and phi.numel() == holo.N
        phi = phi.contiguous()
        V = torch.empty(2 * holo.M, dtype=torch.float32, device=phi.device)
        hot.hot_field(holo.ctx, phi, V)
        ctx.save_for_backward(phi)
        ctx.holo = holo
        return torch.view_as_complex(V.view(holo.M, 2))

    @staticmethod
    def backward(ctx, gV: torch.Tensor):
        (phi,) = ctx.saved_tensors
        holo = ctx.holo
        G = torch.view_as_real(gV.to(torch.complex64).contiguous()).reshape(-1).contiguous()
        grad = torch.empty_like(phi)
        hot.hot_field_adjoint(holo.ctx, phi, G, grad)
        return grad, None


def trap_fields(holo: "hot.Hologram", phi: torch.Tensor) -> torch.Tensor:
    """Complex64 trap fields V (M,) of the phases phi (N,), differentiable in phi."""
    return TrapFields.apply(phi, holo)


def trap_intensity_loss(V: torch.Tensor, beta: float = 10.0) -> torch.Tensor:
    """-sum_m log I_m + beta var(I) with I_m = |V_m|^2 and the population variance."""
    I = V.real ** 2 + V.imag ** 2
    return -torch.log(I).sum() + beta * I.var(correction=0)


class IntensityLoss(torch.autograd.Function):
    """L(phi) = -sum log I + beta var(I) and dL/dphi from one hot_intensity_loss call; backward
    scales the gradient computed with the loss."""

    @staticmethod
    def forward(ctx, phi: torch.Tensor, holo: "hot.Hologram", beta: float) -> torch.Tensor:
        assert phi.is_cuda and phi.dtype == torch.float32 and phi.numel() == holo.N
        phi = phi.contiguous()
        loss = torch.empty(1, dtype=torch.float32, device=phi.device)
        grad = torch.empty_like(phi) if ctx.needs_input_grad[0] else None
        hot.hot_intensity_loss(holo.ctx, phi, beta, loss, grad)
        ctx.save_for_backward(grad if grad is not None else loss)
        return loss[0]

    @staticmethod
    def backward(ctx, gL: torch.Tensor):
        (grad,) = ctx.saved_tensors
        return grad * gL, None, None


def intensity_loss(holo: "hot.Hologram", phi: torch.Tensor, beta: float = 10.0) -> torch.Tensor:
    """-sum_m log I_m + beta var(I) of the traps' intensities for phases phi, differentiable in phi."""
    return IntensityLoss.apply(phi, holo, beta)
