"""The structure the GPU's block coarse solver rests on, checked on the oracle's A_0.

The coarse matrix A_0 = R_0 A R_0^T (Eq. 4) couples coarse nodes up to two coarse rows
apart for B_2 (its functions span three coarse cells) and one row apart for P_1.
Ordered by coarse rows, with s coarse rows to a block (s = 2 for B_2, 1 for P_1, the
last block shorter when the row count is odd), A_0 is block tridiagonal.  Then block
LU

  S_0 = D_0,  S_i = D_i - L_i S_{i-1}^{-1} U_{i-1},  W_i = S_i^{-1}
  forward  y_i = W_i (b_i - L_i y_{i-1})
  backward x_i = y_i - W_i U_i x_{i+1}

solves A_0 x = b exactly in 2m - 1 dependent block products (m blocks).  That is how
the GPU's exact coarse solve handles large coarse spaces.  Checked for MP-1 and MP-2
with a kappa field against numpy.linalg.solve.
"""
import numpy as np
import pytest

from oracle import B2, DIRICHLET, P1, SOMMERFELD, CoarseSpace, Problem
from paper_2408_03571_gb300.inputs import kappa_field


def blocks_of(nc1, s):
    starts = list(range(0, nc1, s))
    return [(a, min(a + s, nc1)) for a in starts]


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
@pytest.mark.parametrize("kind,s", [(B2, 2), (P1, 1)])
def test_coarse_matrix_is_block_tridiagonal_and_block_lu_is_exact(bc, kind, s):
    n, p = 65, 4
    prob = Problem(n, bc, kappa_field(n, 12.0, seed=51))
    cs = CoarseSpace(prob, kind, p)
    A0 = cs.galerkin(prob.assemble_fast())
    nc1 = cs.nc1
    rows = [slice(a * nc1, b * nc1) for a, b in blocks_of(nc1, s)]
    m = len(rows)
    for i in range(m):
        for k in range(m):
            blk = A0[rows[i], rows[k]]
            if abs(i - k) > 1:
                assert np.max(np.abs(blk)) <= 1e-12 * np.max(np.abs(A0))
            elif abs(i - k) == 1:
                assert np.max(np.abs(blk)) > 0
    if s == 2:      # one coarse row per block would not do for B_2
        J = nc1 // 2
        assert np.max(np.abs(A0[J * nc1:(J + 1) * nc1, (J + 2) * nc1:(J + 3) * nc1])) > 0
    D = [A0[rows[i], rows[i]] for i in range(m)]
    L = [None] + [A0[rows[i], rows[i - 1]] for i in range(1, m)]
    U = [A0[rows[i], rows[i + 1]] for i in range(m - 1)] + [None]
    rng = np.random.default_rng(52)
    b = rng.standard_normal(A0.shape[0]) + 1j * rng.standard_normal(A0.shape[0])
    W, y = [], []
    for i in range(m):
        S = D[i] if i == 0 else D[i] - L[i] @ W[i - 1] @ U[i - 1]
        W.append(np.linalg.inv(S))
        bi = b[rows[i]] if i == 0 else b[rows[i]] - L[i] @ y[i - 1]
        y.append(W[i] @ bi)
    x = [None] * m
    x[m - 1] = y[m - 1]
    for i in range(m - 2, -1, -1):
        x[i] = y[i] - W[i] @ (U[i] @ x[i + 1])
    x = np.concatenate(x)
    ref = np.linalg.solve(A0, b)
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
