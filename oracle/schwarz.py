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
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .coarse import CoarseSolver, CoarseSpace
from .decomposition import Decomposition

AS1, AS2, SAS2, SHS2 = "as1", "as2", "sas2", "shs2"


class Schwarz:
    def __init__(self, prob, A, ns: int, overlap: int, kind: str = SHS2,
                 coarse: str | None = "b2", p: int | None = None):
        if kind not in (AS1, AS2, SAS2, SHS2):
            raise ValueError(kind)
        if kind != AS1 and coarse is None:
            raise ValueError("two-level preconditioners need a coarse space")
        self.kind, self.A = kind, A
        self.dec = Decomposition(prob, ns, overlap)
        Ar = A.tocsr()
        self.lu = []
        for s in self.dec.subs:
            Ai = Ar[s.idx][:, s.idx].tocsc()
            # A_i has a symmetric nonzero pattern (Section 2), so the fill-reducing
            # ordering is minimum degree on A^T + A
            self.lu.append(spla.splu(Ai, permc_spec="MMD_AT_PLUS_A"))
        self.coarse = None
        if kind != AS1:
            self.coarse = CoarseSolver(CoarseSpace(prob, coarse, p), Ar)

    def local_sum(self, r: np.ndarray, weighted: bool) -> np.ndarray:
        """sum_i R_i^T (D_i) A_i^{-1} R_i r."""
        out = np.zeros_like(r, dtype=np.complex128)
        for s, lu in zip(self.dec.subs, self.lu):
            y = lu.solve(np.ascontiguousarray(r[s.idx], dtype=np.complex128))
            self.dec.prolong_add(s, y, out, weighted)
        return out

    def apply(self, v: np.ndarray) -> np.ndarray:
        """z = M^{-1} v."""
        if self.kind == AS1:
            return self.local_sum(v, weighted=False)
        q = self.coarse.apply_Q(v)
        if self.kind == AS2:
            return q + self.local_sum(v, weighted=False)
        if self.kind == SAS2:
            return q + self.local_sum(v, weighted=True)
        # SHS2: coarse correction first, then local solves on the deflated residual
        w = v - self.A @ q
        return q + self.local_sum(w, weighted=True)
