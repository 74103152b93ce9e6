"""Oracle: one- and two-level Schwarz preconditioners (Section 3, Eqs. (4)-(6)).

TEST INFRASTRUCTURE ONLY (FP64 CPU restatement, no code shared with the CUDA path).

With Q = R_0^T A_0^{-1} R_0 (A_0 = R_0 A R_0^T) and exact local solves
A_i^{-1} = (R_i A R_i^T)^{-1} done by a sparse direct solver (Section 3):

* AS1  (one-level additive):      M^{-1} = sum_i R_i^T A_i^{-1} R_i
* AS2  (Eq. (4)):                 M^{-1} = Q + sum_i R_i^T A_i^{-1} R_i
* SAS2 (Eq. (5)):                 M^{-1} = Q + sum_i R_i^T D_i A_i^{-1} R_i
* SHS2 (Eq. (6)):                 M^{-1} = Q + (sum_i R_i^T D_i A_i^{-1} R_i)(I - A Q)

The local problems are factorised once with SuperLU (scipy.sparse.linalg.splu,
minimum-degree ordering on A_i^T + A_i, partial pivoting).

Mixed precision (``precision="c64"``): the paper computes in one precision; the
reduced-precision preconditioner of the mixed solver is read as the same
operator with its transfers (R_0, R_0^T, R_i, R_i^T D_i), its deflation
v - A q and its exact local solves applied in complex64 - the input is rounded
to complex64, every product and sum is a complex64 operation - while the
set-up and the coarse solve stay in FP64: each local matrix is factorised by
SuperLU in FP64 once, its factors L and U are rounded to complex64 and the two
triangular solves run in complex64; A_0^{-1} is applied in FP64 (its input
widened from, its output rounded to, complex64).  The result is returned
widened to complex128 for the FP64 flexible GMRES around it.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .coarse import B2, CoarseSolver, CoarseSpace
from .decomposition import Decomposition

AS1, AS2, SAS2, SHS2 = "as1", "as2", "sas2", "shs2"


FP64, C64 = "fp64", "c64"


class MultilevelCoarseSolver:
    """Inexact coarse solve for large coarse spaces (the paper names the exact coarse solve
    as the bottleneck when |G_H| is large, Section 5): A_0^{-1} replaced by one application
    of the two-level Schwarz method SHS2 (Eq. 6) on the coarse grid G_H itself - coarse
    subdomains of G_H with exact local solves of the blocks of A_0 and a B_2 coarse space of
    ratio p0 on G_H with its own exact Galerkin solve.  With a single coarse subdomain it
    is A_0^{-1} exactly (Q_00 + A_0^{-1} (I - A_0 Q_00) = A_0^{-1}).

    inner_tol: None applies M_0^{-1} once (a fixed linear approximation of A_0^{-1});
    a tolerance runs right-preconditioned GMRES on A_0 c' = c with M_0 to that relative
    residual instead (a nonlinear coarse solve: the outer iteration must then be the
    flexible GMRES).  A coarse-of-coarse level is as bound by k H_0 <= 1 as the first
    one (Section 5), so single applications need H_0 small; inner iterations do not."""

    def __init__(self, prob, cs, A0, ns0, ov0: int, p0: int, inner_tol: float | None = None,
                 inner_maxit: int = 200):
        import scipy.sparse as sp
        from .problem import DIRICHLET, Problem
        # G_H as a grid: MP-1 keeps only its interior coarse nodes, so it is the interior of a
        # Dirichlet grid two nodes wider; MP-2 keeps all of them
        n0 = cs.nc1 + 2 if prob.bc == DIRICHLET else cs.nc1
        self.prob0 = Problem(n0, prob.bc, 1.0)
        if self.prob0.N != A0.shape[0]:
            raise ValueError("coarse grid and coarse matrix disagree")
        self.A0 = sp.csr_matrix(A0)
        self.M0 = Schwarz(self.prob0, self.A0, ns0, ov0, SHS2, B2, p0)
        self.inner_tol, self.inner_maxit = inner_tol, inner_maxit
        self.inner_its = []

    def solve(self, c: np.ndarray) -> np.ndarray:
        """The approximation of A_0^{-1} c (FP64)."""
        c = np.asarray(c, dtype=np.complex128)
        if self.inner_tol is None:
            return self.M0.apply(c)
        from .gmres import gmres
        r = gmres(lambda x: self.A0 @ x, self.M0.apply, c, self.inner_tol, self.inner_maxit)
        self.inner_its.append(r.iterations)
        return r.x


class Schwarz:
    def __init__(self, prob, A, ns, overlap: int, kind: str = SHS2,
                 coarse: str | None = "b2", p: int | None = None, precision: str = FP64,
                 scaling: str = "owner", b2_mode: str = "spline", coarse_solve: dict | None = None):
        """coarse_solve: None for the exact coarse solve (dense LU of A_0), or
        dict(ns=, ov=, p=[, inner_tol=]) for the multilevel one (MultilevelCoarseSolver)."""
        if kind not in (AS1, AS2, SAS2, SHS2):
            raise ValueError(kind)
        if kind != AS1 and coarse is None:
            raise ValueError("two-level preconditioners need a coarse space")
        if precision not in (FP64, C64):
            raise ValueError(precision)
        self.kind, self.A, self.precision = kind, A, precision
        self.ct = np.complex128 if precision == FP64 else np.complex64
        self.dec = Decomposition(prob, ns, overlap, scaling)
        Ar = A.tocsr()
        # the operator in the preconditioner's precision (the deflation of SHS2)
        self.Ap = A if precision == FP64 else Ar.astype(self.ct)
        self.lu = []
        self.lu32 = []
        for s in self.dec.subs:
            Ai = Ar[s.idx][:, s.idx].tocsc()
            # A_i has a symmetric nonzero pattern (Section 2), so the fill-reducing
            # ordering is minimum degree on A^T + A
            lu = spla.splu(Ai, permc_spec="MMD_AT_PLUS_A")
            self.lu.append(lu)
            if precision == C64:
                # Pr A_i Pc = L U: the FP64 factors rounded to complex64
                self.lu32.append((lu.L.astype(np.complex64).tocsr(), lu.U.astype(np.complex64).tocsr(),
                                  lu.perm_r, lu.perm_c))
        self.coarse = None
        if kind != AS1:
            self.coarse = CoarseSolver(CoarseSpace(prob, coarse, p, b2_mode), Ar)
            if coarse_solve is not None:
                self.coarse.inner = MultilevelCoarseSolver(prob, self.coarse.cs, self.coarse.A0, coarse_solve["ns"],
                                                           coarse_solve["ov"], coarse_solve["p"],
                                                           coarse_solve.get("inner_tol"))
            if precision == C64:
                self.R0p = self.coarse.cs.R0.astype(np.float32)

    def local_sum(self, r: np.ndarray, weighted: bool) -> np.ndarray:
        """sum_i R_i^T (D_i) A_i^{-1} R_i r, in the preconditioner's precision."""
        out = np.zeros_like(r, dtype=self.ct)
        for k, (s, lu) in enumerate(zip(self.dec.subs, self.lu)):
            if self.precision == C64:
                y = self._solve32(k, np.ascontiguousarray(r[s.idx], dtype=np.complex64))
            else:
                y = lu.solve(np.ascontiguousarray(r[s.idx], dtype=np.complex128))
            if weighted:
                out[s.idx] += s.d.astype(y.real.dtype) * y
            else:
                out[s.idx] += y
        return out

    def _solve32(self, k: int, b: np.ndarray) -> np.ndarray:
        """A_k^{-1} b with the complex64 factors: z = U^{-1} L^{-1} (Pr b), x = Pc z."""
        L, U, perm_r, perm_c = self.lu32[k]
        pb = np.empty_like(b)
        pb[perm_r] = b
        y = spla.spsolve_triangular(L, pb, lower=True, unit_diagonal=True)
        z = spla.spsolve_triangular(U, y, lower=False)
        return z[perm_c]

    def apply_Q(self, v: np.ndarray) -> np.ndarray:
        """Q v = R_0^T A_0^{-1} R_0 v: the transfers in the preconditioner's precision,
        the coarse solve in FP64."""
        if self.precision == FP64:
            return self.coarse.apply_Q(v)
        c = (self.R0p @ v).astype(np.complex128)
        c = self.coarse.solve(c).astype(np.complex64)
        return self.R0p.T @ c

    def apply(self, v: np.ndarray) -> np.ndarray:
        """z = M^{-1} v (complex128 out; computed in complex64 when precision is c64)."""
        v = np.asarray(v).astype(self.ct)
        if self.kind == AS1:
            z = self.local_sum(v, weighted=False)
        else:
            q = self.apply_Q(v)
            if self.kind == AS2:
                z = q + self.local_sum(v, weighted=False)
            elif self.kind == SAS2:
                z = q + self.local_sum(v, weighted=True)
            else:
                # SHS2: coarse correction first, then local solves on the deflated residual
                w = v - self.Ap @ q
                z = q + self.local_sum(w, weighted=True)
        return z.astype(np.complex128)
