"""torch.autograd.Function over qf_energy_grad.

The forward pass runs the whole energy + adjoint-gradient evaluation in libqf
(one C-ABI call) and keeps the gradient; backward scales it by the incoming
gradient.  E(t) = <Phi|U(t)^+ H U(t)|Phi> (Eq. 17-18) with U(t) the dUCC product
of Eq. 19 (or any rotation list with theta_k = coeff_k * t[param_k]).
"""
from __future__ import annotations

import numpy as np
import torch


class EnergyGrad(torch.autograd.Function):
    @staticmethod
    def forward(ctx, t, state, det, ansatz, terms):
        tn = t.detach().to("cpu", torch.float64).numpy()
        e, g = state.energy_grad(int(det), ansatz, np.ascontiguousarray(tn), terms)
        ctx.save_for_backward(torch.as_tensor(g, dtype=t.dtype, device=t.device))
        return torch.tensor(e, dtype=t.dtype, device=t.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None


def energy(t: torch.Tensor, state, det: int, ansatz, terms) -> torch.Tensor:
    """Differentiable energy: `energy(t, ...).backward()` fills t.grad with dE/dt."""
    return EnergyGrad.apply(t, state, det, ansatz, terms)
