"""Oracle: coarse spaces P_1 and B_2 and the Galerkin coarse matrix (Section 4).

TEST INFRASTRUCTURE ONLY (FP64 CPU restatement, no code shared with the CUDA path).

The coarse mesh G_H has nodes X_I = I H, I = 0 .. 1/H, with ``p = H/h`` an
integer >= 2 dividing n-1.  A row of R_0 is a coarse basis function sampled at
the fine unknowns; in 2-D it is the tensor product phi_I(x) phi_J(y).

* P_1 (Section 4, "linear coarse basis"): the hat function
  ``phi_I(x) = max(0, 1 - |x - X_I| / H)``.
* B_2 (Section 4, Eq. (7)): the paper prints the restriction for H = 2h as the
  weights (1, 4, 6, 4, 1)/8 around fine node m = 2i - 1.  Those are the values of
  the uniform quadratic B-spline with knot spacing H centred at X_I, sampled at
  the fine nodes: ``phi_I(x) = B2((x - X_I)/H + 3/2)`` with the cardinal
  quadratic B-spline B2 on [0, 3].  That function is used for every p (for
  p = 2 it reproduces Eq. (7) exactly; tests check this).
* Alternative reading of B_2 for H = 2^m h (``b2_mode="composed"``): Eq. (7)'s
  restriction from spacing s to 2s, weights (1, 4, 6, 4, 1)/8 around the fine
  node under each coarse node, applied m times (coarse to fine: level by level),
  each level on the full node set of its grid.  For m = 1 both readings coincide.
* Fine nodes outside the unknowns are dropped (truncation at the boundary).
  MP-1 drops the coarse nodes on the boundary (their functions would carry the
  eliminated Dirichlet values); MP-2 keeps all (1/H + 1)^2 coarse nodes.
* Prolongation is R_0^T (Section 4); the coarse matrix is A_0 = R_0 A R_0^T
  (Eq. (4)), solved exactly (dense LU with partial pivoting here).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .problem import DIRICHLET

P1 = "p1"
B2 = "b2"


def bspline2(t):
    """Cardinal quadratic B-spline on [0, 3] (zero outside)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    a = (t >= 0) & (t < 1)
    b = (t >= 1) & (t < 2)
    c = (t >= 2) & (t <= 3)
    out[a] = 0.5 * t[a] ** 2
    out[b] = 0.5 * (-2.0 * t[b] ** 2 + 6.0 * t[b] - 3.0)
    out[c] = 0.5 * (3.0 - t[c]) ** 2
    return out


def hat(t):
    """Linear hat on [-1, 1]."""
    t = np.asarray(t, dtype=np.float64)
    return np.maximum(0.0, 1.0 - np.abs(t))


SPLINE, COMPOSED = "spline", "composed"


def eq7_level(nf: int) -> np.ndarray:
    """Eq. (7)'s restriction from nf nodes (spacing s) to (nf - 1)/2 + 1 nodes (spacing 2s),
    all nodes of both grids: row I has (1, 4, 6, 4, 1)/8 on fine nodes 2I - 2 .. 2I + 2."""
    nc = (nf - 1) // 2 + 1
    R = np.zeros((nc, nf))
    for I in range(nc):
        for d, wgt in zip(range(-2, 3), (1.0, 4.0, 6.0, 4.0, 1.0)):
            if 0 <= 2 * I + d < nf:
                R[I, 2 * I + d] = wgt / 8.0
    return R


def basis_1d(kind: str, n: int, p: int, keep_ends: bool, b2_mode: str = SPLINE) -> np.ndarray:
    """(number of coarse nodes) x n matrix of phi_I(x_i) over all fine nodes i."""
    if p < 2 or (n - 1) % p != 0:
        raise ValueError("coarse ratio p = H/h must be >= 2 and divide n-1")
    if kind == B2 and b2_mode == COMPOSED:
        m = int(round(np.log2(p)))
        if 2 ** m != p:
            raise ValueError("the composed B2 needs H/h a power of two")
        W = np.eye(n)
        nf = n
        for _ in range(m):
            W = eq7_level(nf) @ W
            nf = (nf - 1) // 2 + 1
        return W if keep_ends else W[1:-1]
    if b2_mode not in (SPLINE, COMPOSED):
        raise ValueError(b2_mode)
    nc = (n - 1) // p + 1
    H = p / (n - 1)
    x = np.arange(n) / (n - 1)
    I0, I1 = (0, nc) if keep_ends else (1, nc - 1)
    rows = []
    for I in range(I0, I1):
        XI = I * H
        if kind == B2:
            rows.append(bspline2((x - XI) / H + 1.5))
        elif kind == P1:
            rows.append(hat((x - XI) / H))
        else:
            raise ValueError(kind)
    return np.array(rows)


class CoarseSpace:
    def __init__(self, prob, kind: str, p: int, b2_mode: str = SPLINE):
        self.kind, self.p = kind, p
        keep = prob.bc != DIRICHLET
        W = basis_1d(kind, prob.n, p, keep, b2_mode)[:, prob.lo:prob.hi + 1]   # truncate to unknowns
        self.W1 = W
        self.nc1 = W.shape[0]
        # coarse index J*nc1 + I  <->  phi_I(x) phi_J(y); fine index j*m + i
        self.R0 = sp.csr_matrix(sp.kron(sp.csr_matrix(W), sp.csr_matrix(W)))
        self.Nc = self.R0.shape[0]

    def galerkin(self, A: sp.spmatrix) -> np.ndarray:
        """Dense A_0 = R_0 A R_0^T (Eq. (4))."""
        return (self.R0 @ A @ self.R0.T).toarray()


class CoarseSolver:
    """Exact coarse solve with A_0 = R_0 A R_0^T by dense LU with partial pivoting."""

    def __init__(self, cs: CoarseSpace, A):
        self.cs = cs
        self.A0 = cs.galerkin(A)
        self.lu = sla.lu_factor(self.A0)
        self.inner = None           # a multilevel solver standing in for A_0^{-1} (see schwarz.py)

    def solve(self, c: np.ndarray) -> np.ndarray:
        """A_0^{-1} c (FP64), or its multilevel approximation when one is set."""
        if self.inner is not None:
            return self.inner.solve(c)
        return sla.lu_solve(self.lu, np.asarray(c, dtype=np.complex128))

    def apply_Q(self, v: np.ndarray) -> np.ndarray:
        """Q v = R_0^T A_0^{-1} R_0 v."""
        c = self.cs.R0 @ v
        c = self.solve(c)
        return self.cs.R0.T @ c
