"""Oracle: adjoint solve and the gradient of a receiver misfit w.r.t. kappa = k^2.

TEST INFRASTRUCTURE ONLY (FP64 CPU restatement, no code shared with the CUDA path).
The paper has no counterpart; this is the differentiation layer added on top
of its solver.  Derivation (A depends on the real field kappa through its
diagonal only, see ``Problem.ddiag_dkappa``):

  A(kappa) u = f,   L = 1/2 sum_{r in receivers} |u_r - t_r|^2
  dL/dkappa_j = Re( (P(u - t))^H du/dkappa_j ),   A du/dkappa_j = -(dA/dkappa_j) u
             = -Re( lambda^H (dA/dkappa_j) u ),    conj(A) lambda = P(u - t)
  Since A = A^T, conj(A) lambda = g is the same as A mu = conj(g), mu = conj(lambda), so
  dL/dkappa_j = -Re( mu_j * dA_jj/dkappa_j * u_j ).
"""
from __future__ import annotations

import numpy as np

from .gmres import gmres


def misfit_residual(u: np.ndarray, target: np.ndarray, receivers: np.ndarray) -> np.ndarray:
    """g = P(u - t): zero except on the receiver unknowns."""
    g = np.zeros_like(u, dtype=np.complex128)
    g[receivers] = u[receivers] - target[receivers]
    return g


def loss(u: np.ndarray, target: np.ndarray, receivers: np.ndarray) -> float:
    d = u[receivers] - target[receivers]
    return 0.5 * float(np.sum(np.abs(d) ** 2))


def adjoint_solve(A, M_apply, g: np.ndarray, tol: float, maxit: int):
    """Solve conj(A) lambda = g with the same preconditioned GMRES (via A mu = conj(g))."""
    res = gmres(lambda x: A @ x, M_apply, np.conj(g), tol, maxit)
    lam = np.conj(res.x)
    return lam, res


def kappa_gradient(dA_dkappa: np.ndarray, u: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """dL/dkappa_j = -Re(conj(lambda_j) dA_jj/dkappa_j u_j) over the unknowns."""
    return -np.real(np.conj(lam) * dA_dkappa * u)
