"""PyTorch autograd wrappers around libtetra (both directions run in the CUDA
kernels; PyTorch only holds the tensors and the graph).

* ``TetraDosFn``: bin-mode DOS (Eqs. (8)-(9) averaged over bins) with its
  adjoint ``tetra_dos_backward`` -> gradients for band energies and orbital
  weights.
* ``TetraEigFn``: band structure of a tight-binding model (``tetra_eig``) with
  its adjoint ``tetra_eig_backward`` -> gradients for the hopping parameters.
* ``model_dos``: parameters -> bin DOS through both, for fitting hoppings to a
  target DOS.
"""
from __future__ import annotations

import torch

from . import Plan


class TetraDosFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, w, edges, plan: Plan):
        if plan.mode != "bin":
            raise ValueError("TetraDosFn needs a bin-mode plan")
        dos = plan.dos(eps, w, edges)
        ctx.save_for_backward(eps, w, edges)
        ctx.plan = plan
        return dos

    @staticmethod
    def backward(ctx, grad_dos):
        eps, w, edges = ctx.saved_tensors
        ge, gw = ctx.plan.dos_backward(eps, w, edges, grad_dos.contiguous().float())
        return ge, gw.to(w.dtype), None, None


class TetraEigFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, R, plan: Plan):
        eps, w = plan.eig(params, R)
        ctx.save_for_backward(params, R)
        ctx.plan = plan
        return eps, w

    @staticmethod
    def backward(ctx, grad_eps, grad_w):
        params, R = ctx.saved_tensors
        plan = ctx.plan
        eps_shape, w_shape = plan.empty_inputs()
        if grad_eps is None:
            grad_eps = torch.zeros_like(eps_shape)
        if grad_w is None:
            grad_w = torch.zeros(w_shape.shape, dtype=torch.float32, device=params.device)
        g = plan.eig_backward(params, R, grad_eps.contiguous().float(),
                              grad_w.contiguous().float())
        return g, None, None


def model_dos(params, R, edges, plan: Plan):
    """Bin-averaged orbital DOS of the model with parameters ``params``
    (differentiable with respect to ``params``)."""
    eps, w = TetraEigFn.apply(params, R, plan)
    return TetraDosFn.apply(eps, w, edges, plan)
