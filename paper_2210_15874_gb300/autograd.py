"""torch.autograd wrapper of the noisy-QAOA ensemble energy.

``qaoa_energy(gammas, betas, batch, edges, **noise)`` returns the ensemble mean
<C> as a 0-d tensor; its backward calls the library's adjoint kernels
(qn_grad) for d<C>/d gamma and d<C>/d beta.  Forward and backward both run on
the GPU through the C ABI; the wrapper only marshals tensors.  Pauli-only noise
is required for the backward pass (damping makes trajectories non-unitary).

qn_grad differentiates the circuit a handle ran last.  When the same Batch has
run again between a forward and its backward (two energies on one Batch summed
into one loss, or a forward followed by other runs), the backward first re-runs
its own forward's circuit on the handle -- the same angles, graph, noise and
seed give the same trajectories -- so every backward returns the gradient at
the angles of its own forward.  That re-run replaces the handle's last results.
"""
from __future__ import annotations

import numpy as np
import torch

from . import qn


class _QaoaEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gammas, betas, batch, edges, noise):
        g = gammas.detach().cpu().numpy().astype(np.float64)
        b = betas.detach().cpu().numpy().astype(np.float64)
        batch.run_qaoa(edges, g, b, **noise)
        mean, _ = batch.expectation()
        ctx.batch = batch
        ctx.run = (edges, g, b, dict(noise))
        ctx.generation = batch.generation
        ctx.dtype, ctx.device = gammas.dtype, gammas.device
        return torch.tensor(mean, dtype=gammas.dtype, device=gammas.device)

    @staticmethod
    def backward(ctx, grad_out):
        batch = ctx.batch
        if batch.generation != ctx.generation:
            edges, g, b, noise = ctx.run
            batch.run_qaoa(edges, g, b, **noise)
        dg, db = batch.grad()
        scale = grad_out.detach().to("cpu", torch.float64).item()
        tg = torch.tensor(dg * scale, dtype=ctx.dtype, device=ctx.device)
        tb = torch.tensor(db * scale, dtype=ctx.dtype, device=ctx.device)
        return tg, tb, None, None, None


def qaoa_energy(gammas: torch.Tensor, betas: torch.Tensor, batch: "qn.Batch", edges, **noise) -> torch.Tensor:
    """Ensemble <C> of the noisy QAOA circuit, differentiable in gammas and betas."""
    return _QaoaEnergy.apply(gammas, betas, batch, edges, noise)
