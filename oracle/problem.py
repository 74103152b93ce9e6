"""Oracle: the discrete model problems MP-1 / MP-2 (Section 2, Eqs. (1)-(3)).

TEST INFRASTRUCTURE ONLY.  Plain, slow FP64 CPU restatement; it shares no code
with the CUDA path and must never be imported by the product package.

The unknown vector is the list of unknown grid nodes in lexicographic order
(x index fastest).  MP-1 (Dirichlet, Eq. (1)): the interior nodes; the boundary
values are zero and are eliminated.  MP-2 (Sommerfeld, Eq. (2)): every node.

Assembly of ``A u = f`` (Eq. (3)), second-order finite differences:

* interior node: ``(4 u_P - u_E - u_W - u_N - u_S) / h^2 - kappa_P u_P``;
* Sommerfeld boundary node: the normal derivative in ``du/dn - i k u = 0`` is
  taken by a central difference through a ghost node outside the square,
  ``u_ghost = u_inward + 2 i h k u_P``, which is substituted into the 5-point
  row.  The row is then multiplied by 1/2 on an edge and by 1/4 at a corner
  (a corner has a ghost in both directions), which makes ``A`` symmetric as
  Section 2 states.  With ``k = sqrt(kappa_P)`` this gives
    edge:   diag 2/h^2 - kappa/2 - i k/h, inward neighbour -1/h^2,
            neighbours along the edge -1/(2 h^2);
    corner: diag 1/h^2 - kappa/4 - i k/h, both neighbours -1/(2 h^2).
  The right-hand side of a scaled row is scaled the same way; the API takes
  ``f`` as the right-hand side of the scaled (symmetric) system.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

DIRICHLET = "dirichlet"   # MP-1
SOMMERFELD = "sommerfeld"  # MP-2


class Problem:
    """Grid, boundary type and squared wavenumber of one model problem."""

    def __init__(self, n: int, bc: str, kappa):
        if n < 3 or n % 2 != 1:
            raise ValueError("n must be odd and >= 3")
        if bc not in (DIRICHLET, SOMMERFELD):
            raise ValueError(bc)
        self.n = n
        self.h = 1.0 / (n - 1)
        self.bc = bc
        kap = np.asarray(kappa, dtype=np.float64)
        self.kappa = np.full((n, n), float(kap)) if kap.ndim == 0 else kap.copy()
        if self.kappa.shape != (n, n):
            raise ValueError("kappa must be scalar or (n, n)")
        lo, hi = (1, n - 2) if bc == DIRICHLET else (0, n - 1)
        self.lo, self.hi = lo, hi            # inclusive range of unknown indices per axis
        self.m = hi - lo + 1                  # unknowns per axis
        self.N = self.m * self.m

    # --- index maps -------------------------------------------------------
    def index(self, i, j):
        """Unknown index of grid node (i, j) (x index i, y index j)."""
        return (j - self.lo) * self.m + (i - self.lo)

    def is_unknown(self, i, j):
        return self.lo <= i <= self.hi and self.lo <= j <= self.hi

    def grid_to_vec(self, g: np.ndarray) -> np.ndarray:
        """(n, n) or (..., n, n) grid array -> unknown vector(s)."""
        s = g[..., self.lo:self.hi + 1, self.lo:self.hi + 1]
        return s.reshape(s.shape[:-2] + (self.N,)).copy()

    def vec_to_grid(self, v: np.ndarray) -> np.ndarray:
        """Unknown vector(s) -> (n, n) grid array(s), zero on eliminated nodes."""
        v = np.asarray(v)
        out = np.zeros(v.shape[:-1] + (self.n, self.n), dtype=np.result_type(v, np.complex128))
        out[..., self.lo:self.hi + 1, self.lo:self.hi + 1] = v.reshape(v.shape[:-1] + (self.m, self.m))
        return out

    # --- node classification (MP-2) --------------------------------------
    def boundary_count(self, i, j):
        """Number of boundary lines (0, 1 or 2) the node lies on."""
        n = self.n
        return int(i in (0, n - 1)) + int(j in (0, n - 1))

    def diag_entry(self, i, j):
        """Diagonal entry A_PP of the node's row."""
        h, kap = self.h, self.kappa[j, i]
        if self.bc == DIRICHLET:
            return complex(4.0 / h**2 - kap)
        nb = self.boundary_count(i, j)
        if nb == 0:
            return complex(4.0 / h**2 - kap)
        k = np.sqrt(kap)
        if nb == 1:
            return complex(2.0 / h**2 - kap / 2.0, -k / h)
        return complex(1.0 / h**2 - kap / 4.0, -k / h)

    def ddiag_dkappa(self, i, j):
        """d A_PP / d kappa_P (only the node's own diagonal depends on kappa_P)."""
        h, kap = self.h, self.kappa[j, i]
        if self.bc == DIRICHLET:
            return complex(-1.0)
        nb = self.boundary_count(i, j)
        if nb == 0:
            return complex(-1.0)
        dk = 1.0 / (2.0 * np.sqrt(kap))   # d sqrt(kappa) / d kappa
        if nb == 1:
            return complex(-0.5, -dk / h)
        return complex(-0.25, -dk / h)

    def offdiag_entry(self, i, j, di, dj):
        """Coupling of node (i, j) to its neighbour (i+di, j+dj) (an unknown)."""
        h = self.h
        if self.bc == DIRICHLET:
            return -1.0 / h**2
        n = self.n
        on_x_edge = i in (0, n - 1)   # node on a vertical boundary line
        on_y_edge = j in (0, n - 1)   # node on a horizontal boundary line
        nb = int(on_x_edge) + int(on_y_edge)
        if nb == 0:
            return -1.0 / h**2
        if nb == 2:
            return -0.5 / h**2
        # edge node: the neighbour across the edge normal is "inward" (weight 1
        # after halving the doubled ghost coupling); neighbours along the edge
        # carry the halved weight.
        if on_x_edge:
            return -1.0 / h**2 if di != 0 else -0.5 / h**2
        return -1.0 / h**2 if dj != 0 else -0.5 / h**2

    # --- assembly ----------------------------------------------------------
    def assemble(self) -> sp.csr_matrix:
        """Sparse A over the unknowns, assembled row by row from the rules above."""
        rows, cols, vals = [], [], []
        for j in range(self.lo, self.hi + 1):
            for i in range(self.lo, self.hi + 1):
                p = self.index(i, j)
                rows.append(p); cols.append(p); vals.append(self.diag_entry(i, j))
                for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                    a, b = i + di, j + dj
                    if self.is_unknown(a, b):
                        rows.append(p); cols.append(self.index(a, b))
                        vals.append(complex(self.offdiag_entry(i, j, di, dj)))
        return sp.csr_matrix((np.array(vals, dtype=np.complex128), (rows, cols)),
                             shape=(self.N, self.N))

    def assemble_fast(self) -> sp.csr_matrix:
        """Same matrix as :meth:`assemble`, built with array operations for large n.

        Tests check that the two agree exactly on small grids.
        """
        n, h, lo, hi, m = self.n, self.h, self.lo, self.hi, self.m
        jj, ii = np.meshgrid(np.arange(lo, hi + 1), np.arange(lo, hi + 1), indexing="ij")
        ii = ii.ravel(); jj = jj.ravel()
        p = (jj - lo) * m + (ii - lo)
        kap = self.kappa[jj, ii]
        if self.bc == DIRICHLET:
            nb = np.zeros_like(ii)
        else:
            nb = (ii == 0).astype(int) + (ii == n - 1) + (jj == 0) + (jj == n - 1)
        diag = np.where(nb == 0, 4.0 / h**2 - kap,
                        np.where(nb == 1, 2.0 / h**2 - kap / 2.0, 1.0 / h**2 - kap / 4.0)).astype(np.complex128)
        if self.bc == SOMMERFELD:
            diag = diag - 1j * np.where(nb > 0, np.sqrt(kap) / h, 0.0)
        rows = [p]; cols = [p]; vals = [diag]
        on_x = (ii == 0) | (ii == n - 1)
        on_y = (jj == 0) | (jj == n - 1)
        for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            a, b = ii + di, jj + dj
            ok = (a >= lo) & (a <= hi) & (b >= lo) & (b <= hi)
            w = np.full(ii.shape, -1.0 / h**2)
            if self.bc == SOMMERFELD:
                corner = on_x & on_y
                edge_x = on_x & ~on_y
                edge_y = on_y & ~on_x
                w = np.where(corner, -0.5 / h**2, w)
                if di != 0:
                    w = np.where(edge_y, -0.5 / h**2, w)   # along a horizontal edge
                else:
                    w = np.where(edge_x, -0.5 / h**2, w)   # along a vertical edge
            rows.append(p[ok]); cols.append(((b - lo) * m + (a - lo))[ok]); vals.append(w[ok].astype(np.complex128))
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.N, self.N))

    def dA_dkappa(self) -> np.ndarray:
        """Vector of d A_PP / d kappa_P over the unknowns."""
        out = np.empty(self.N, dtype=np.complex128)
        for j in range(self.lo, self.hi + 1):
            for i in range(self.lo, self.hi + 1):
                out[self.index(i, j)] = self.ddiag_dkappa(i, j)
        return out
