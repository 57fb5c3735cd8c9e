"""Differentiable free energy E(m; Ms0, A0, D0, Ku, chi) as a torch.autograd.Function.

Forward and backward both call mmc_energy_grad (hand-written CUDA kernels);
the backward recomputes the demag convolution instead of storing the field.
"""
from __future__ import annotations

import numpy as np
import torch


class Energy(torch.autograd.Function):
    """E = Energy.apply(m, params, engine, chain)

    m: CUDA tensor (ncell, 3), float32 or float64, natural cell order.
    params: tensor of 5 values (Ms0 [A/m], A0 [J/m], D0 [J/m^2], Ku [J/m^3], chi [1/T]).
    engine: an MMC context whose chain `chain` defines mesh, cell size, T, field.
    Returns the total energy (J) as a 0-dim tensor of m's dtype.
    """

    @staticmethod
    def forward(ctx, m, params, engine, chain=0):
        p = params.detach().to("cpu", torch.float64).numpy()
        E, _, _ = engine.energy_grad(m.detach().contiguous(), params=p, chain=chain, grad=False)
        ctx.save_for_backward(m, params)
        ctx.engine = engine
        ctx.chain = chain
        return torch.tensor(E[0], dtype=m.dtype, device=m.device)

    @staticmethod
    def backward(ctx, gE):
        m, params = ctx.saved_tensors
        p = params.detach().to("cpu", torch.float64).numpy()
        _, dEdm, dEdp = ctx.engine.energy_grad(m.detach().contiguous(), params=p, chain=ctx.chain, grad=True)
        gm = gE.to(m.dtype) * dEdm if ctx.needs_input_grad[0] else None
        gp = None
        if ctx.needs_input_grad[1]:
            gp = gE.to(params.dtype).to(params.device) * torch.tensor(np.asarray(dEdp), dtype=params.dtype,
                                                                   device=params.device)
        return gm, gp, None, None


def energy(engine, m, params, chain=0):
    return Energy.apply(m, params, engine, chain)
