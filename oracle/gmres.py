"""Oracle: right-preconditioned GMRES and flexible GMRES (Section 5).

TEST INFRASTRUCTURE ONLY (FP64 CPU restatement, no code shared with the CUDA path).

Section 5 runs GMRES (Saad and Schultz) with a relative tolerance and an
iteration cap.  The paper does not say which side the preconditioner is on;
this oracle uses right preconditioning, so the residual GMRES minimises is the
true residual of the original system:

  x_0 = 0, r_0 = f, beta = ||f||_2, v_0 = f / beta
  for j = 0, 1, ...:
      z_j = M^{-1} v_j                      (stored as Z for the flexible variant)
      w   = A z_j
      modified Gram-Schmidt: h_ij = <v_i, w>, w -= h_ij v_i   (i = 0..j)
      h_{j+1,j} = ||w||,  v_{j+1} = w / h_{j+1,j}
      complex Givens rotations reduce H to upper triangular; the last entry of
      the rotated right-hand side beta e_1 is the residual norm
      stop when |g_{j+1}| <= tol * ||f||_2 or j+1 = maxit
  y = argmin ||beta e_1 - H y||,  x = M^{-1}(V y)  (or x = Z y, flexible).

The iteration count is the number of Arnoldi steps taken.

Alternative reading (``side="left"``, as MATLAB's gmres applies a preconditioner
given to it): GMRES on M^{-1} A x = M^{-1} f, i.e. v_0 = M^{-1} f / ||M^{-1} f||,
w = M^{-1} A v_j, stop when the preconditioned residual estimate
|g_{j+1}| <= tol ||M^{-1} f||, and x = V y.
"""
from __future__ import annotations

import numpy as np


class GmresResult:
    def __init__(self, x, iterations, converged, resid_hist, relres_true):
        self.x = x
        self.iterations = iterations
        self.converged = converged
        self.resid_hist = resid_hist          # |g_{j+1}| / ||f|| after each step
        self.relres_true = relres_true


def givens(a: complex, b: complex):
    """c (real), s (complex) with [[c, s], [-conj(s), c]] [a, b]^T = [r, 0]^T."""
    aa, bb = abs(a), abs(b)
    if bb == 0.0:
        return 1.0, 0.0 + 0.0j
    if aa == 0.0:
        return 0.0, np.conj(b) / bb
    rho = np.hypot(aa, bb)
    return aa / rho, (a / aa) * np.conj(b) / rho


def gmres(A_apply, M_apply, f: np.ndarray, tol: float, maxit: int,
          flexible: bool = False, A_true=None, side: str = "right") -> GmresResult:
    if side not in ("right", "left"):
        raise ValueError(side)
    left = side == "left"
    f = np.asarray(f, dtype=np.complex128)
    N = f.shape[0]
    f_true = f
    if left:
        f = M_apply(f)
    beta = np.linalg.norm(f)
    if beta == 0.0:
        return GmresResult(np.zeros(N, np.complex128), 0, True, [], 0.0)
    V = [f / beta]
    Z = []
    H = np.zeros((maxit + 1, maxit), dtype=np.complex128)
    cs = np.zeros(maxit)
    sn = np.zeros(maxit, dtype=np.complex128)
    g = np.zeros(maxit + 1, dtype=np.complex128)
    g[0] = beta
    hist = []
    converged = False
    m = 0
    for j in range(maxit):
        if left:
            w = M_apply(A_apply(V[j]))
        else:
            z = M_apply(V[j])
            if flexible:
                Z.append(z)
            w = A_apply(z)
        for i in range(j + 1):                       # modified Gram-Schmidt
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        for i in range(j):                           # previous rotations on column j
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        c, s = givens(H[j, j], H[j + 1, j])
        cs[j], sn[j] = c, s
        H[j, j] = c * H[j, j] + s * H[j + 1, j]
        H[j + 1, j] = 0.0
        g[j + 1] = -np.conj(s) * g[j]
        g[j] = c * g[j]
        m = j + 1
        hist.append(abs(g[j + 1]) / beta)
        if abs(g[j + 1]) <= tol * beta:
            converged = True
            break
        hnext = np.linalg.norm(w)
        if hnext == 0.0:                             # happy breakdown: exact solution
            converged = True
            break
        V.append(w / hnext)
    # back substitution on the m x m upper-triangular system
    y = np.zeros(m, dtype=np.complex128)
    for i in range(m - 1, -1, -1):
        y[i] = (g[i] - H[i, i + 1:m] @ y[i + 1:m]) / H[i, i]
    if left:
        x = sum(y[i] * V[i] for i in range(m))
    elif flexible:
        x = sum(y[i] * Z[i] for i in range(m))
    else:
        x = M_apply(sum(y[i] * V[i] for i in range(m)))
    Atr = A_true if A_true is not None else A_apply
    relres = np.linalg.norm(f_true - Atr(x)) / np.linalg.norm(f_true)
    return GmresResult(x, m, converged, hist, relres)
