"""Differentiable Helmholtz solve: u = A(kappa)^{-1} f with gradients w.r.t. the
squared-wavenumber field kappa and the right-hand side f.

The forward pass factorises the Schwarz preconditioner for the given kappa and
runs preconditioned GMRES (Sections 3-5); the backward pass runs the adjoint
solve conj(A) lambda = grad_u with the same factorisation (A = A^T, Section 2)
and the gradient kernel.  With PyTorch's convention for complex tensors
(grad_u = 2 dL/d conj(u) for a real loss L):

    dL/dkappa_j = -Re( conj(lambda_j) * dA_jj/dkappa_j * u_j ),   dL/df = lambda.

Everything runs in libhzs.so; this module only wires it into autograd.  The
paper has no differentiation layer.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import hzs


@dataclass(frozen=True)
class SolverConfig:
    bc: int = hzs.SOMMERFELD
    nsub: int = 16
    overlap: int = 2
    kind: int = hzs.SHS2
    coarse: int = hzs.COARSE_B2
    coarse_ratio: int = 32
    precision: int = hzs.FP64
    tol: float = 1e-6
    adjoint_tol: float | None = None      # default: tol
    maxit: int = 1000


class HelmholtzSolve(torch.autograd.Function):
    """u = HelmholtzSolve.apply(kappa, f, cfg) with kappa (n, n) float64 and f (n, n) complex128 on CUDA."""

    @staticmethod
    def forward(ctx, kappa: torch.Tensor, f: torch.Tensor, cfg: SolverConfig):
        n = kappa.shape[-1]
        kappa = kappa.detach().contiguous()
        grid = hzs.Grid(n, cfg.bc, kappa=kappa, nsub=cfg.nsub, overlap=cfg.overlap)
        P = hzs.Preconditioner(grid, cfg.kind, cfg.coarse, cfg.coarse_ratio, cfg.precision, dedup_tiles=False)
        u, info = P.solve(f.detach().contiguous(), tol=cfg.tol, maxit=cfg.maxit)
        if not info[0].converged:
            raise hzs.HzsError(hzs.NOT_CONVERGED, f"forward solve did not converge: {info[0]}")
        ctx.grid, ctx.P, ctx.cfg = grid, P, cfg
        ctx.info = info[0]
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, grad_u: torch.Tensor):
        (u,) = ctx.saved_tensors
        P, cfg = ctx.P, ctx.cfg
        tol = cfg.adjoint_tol if cfg.adjoint_tol is not None else cfg.tol
        lam, info = P.adjoint_solve(grad_u.contiguous(), tol=tol, maxit=cfg.maxit)
        if not info[0].converged:
            raise hzs.HzsError(hzs.NOT_CONVERGED, f"adjoint solve did not converge: {info[0]}")
        grad_kappa = P.kappa_gradient(u, lam) if ctx.needs_input_grad[0] else None
        grad_f = lam if ctx.needs_input_grad[1] else None
        P.close()
        ctx.grid.close()
        return grad_kappa, grad_f, None


def solve(kappa: torch.Tensor, f: torch.Tensor, cfg: SolverConfig = SolverConfig()) -> torch.Tensor:
    """Differentiable u = A(kappa)^{-1} f."""
    return HelmholtzSolve.apply(kappa, f, cfg)
