"""Gradient-based tuning of the 4th-kind Chebyshev weights (beta_i of Sec. 2.3, Table 5).

``CycleErrorRatio`` is a torch.autograd.Function around ``chebmg_cycle_error_grad``: its
forward value is f = mean_q ||(I - B A)^steps e0_q||^2 / ||e0_q||^2 (B one V-cycle with the
given weights and lambda_max scale) and its backward returns the exact gradient that the
library computes with the transposed (adjoint) V-cycle on the GPU.  ``tune_weights`` runs Adam
on (beta_1..beta_k, s) from a starting point, e.g. the plain 4th kind (beta = 1), so the result
can be set beside the paper's optimized weights.
"""
from __future__ import annotations

import torch

from . import chebmg_cycle_error_grad


class CycleErrorRatio(torch.autograd.Function):
    """f(betas, scale) for a fixed context and fixed initial errors E0 (rows, on the GPU)."""

    @staticmethod
    def forward(ctx, betas, scale, solver_ctx, E0, steps):
        f, gb, gs, _ = chebmg_cycle_error_grad(solver_ctx, E0, [float(v) for v in betas.detach().cpu()],
                                               float(scale.detach().cpu()), steps)
        ctx.save_for_backward(torch.tensor(gb, dtype=torch.float64), torch.tensor(gs, dtype=torch.float64))
        return torch.tensor(f, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gout):
        gb, gs = ctx.saved_tensors
        return gout * gb.to(gout.device), gout * gs.to(gout.device), None, None, None


def error_ratio(solver_ctx, E0, betas, scale, steps=3):
    """Differentiable f as a CPU scalar tensor (betas: tensor (k,), scale: tensor ())."""
    return CycleErrorRatio.apply(betas, scale, solver_ctx, E0, steps)


def tune_weights(solver_ctx, E0, betas0, scale0=1.0, steps=3, iters=200, lr=0.01, tune_scale=True):
    """Adam on the weights (and the lambda_max scale).  Returns the final (betas, scale) and the
    history of f values (one per step, before the update)."""
    betas = torch.tensor([float(v) for v in betas0], dtype=torch.float64, requires_grad=True)
    scale = torch.tensor(float(scale0), dtype=torch.float64, requires_grad=tune_scale)
    params = [betas] + ([scale] if tune_scale else [])
    opt = torch.optim.Adam(params, lr=lr)
    hist = []
    for _ in range(iters):
        opt.zero_grad()
        f = error_ratio(solver_ctx, E0, betas, scale, steps)
        f.backward()
        opt.step()
        hist.append(float(f.detach()))
        with torch.no_grad():
            scale.clamp_(min=0.05)
    return betas.detach().clone(), float(scale.detach()), hist
