"""torch.autograd bridge: x = K(lambda, mu, rho)^{-1} q with adjoint-state gradients.

Forward runs ehs_fgmres_solve; backward runs ehs_adjoint_solve on the
incoming gradient and ehs_gradient for the medium (the adjoint-state method
behind frequency-domain full-waveform inversion).  PyTorch hands a complex
output the gradient g = dL/dRe(x) + i dL/dIm(x) (twice the conjugate
Wirtinger derivative), so that dL = Re(g^H dx); hence
    w = K^{-H} g,  grad_q = w,  dL/dm = -Re(w^H dK/dm x).
All arithmetic runs in libehs.so; this module only moves tensors.

The solver context built by the forward pass lives as long as the autograd
graph that holds it (it is released with the graph, when the last reference to
the output goes away), so backward may run more than once with
retain_graph=True.
"""
from __future__ import annotations

import torch

from . import ehs


class ElasticHelmholtzSolve(torch.autograd.Function):
    """x = solve(lam, mu, rho, q); lam, mu, rho: float64 (nmedia, *grid) CUDA or
    CPU tensors; q: complex128 CUDA tensor (nmedia * nrhs, d+1, *grid)."""

    @staticmethod
    def forward(ctx, lam, mu, rho, q, omega, h, abl_cells, solver_kw):
        S = ehs.Solver(lam.detach().cpu().numpy(), mu.detach().cpu().numpy(), rho.detach().cpu().numpy(),
                       omega, h, abl_cells, **(solver_kw or {}))
        x = torch.zeros_like(q)
        S.fgmres_solve(q.detach().contiguous(), x)
        ctx.S = S
        ctx.mdev = lam.device
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        S = ctx.S
        w = torch.zeros_like(x)
        S.adjoint_solve(gx.contiguous(), w)
        gl, gm, gr = S.gradient(x, w)
        need = ctx.needs_input_grad
        to = lambda t: t.to(ctx.mdev)
        return (to(gl) if need[0] else None, to(gm) if need[1] else None, to(gr) if need[2] else None,
                w if need[3] else None, None, None, None, None)


def solve(lam, mu, rho, q, omega, h=1.0, abl_cells=10, **solver_kw):
    """Differentiable elastic Helmholtz solve (see ElasticHelmholtzSolve)."""
    return ElasticHelmholtzSolve.apply(lam, mu, rho, q, omega, h, abl_cells, solver_kw)
