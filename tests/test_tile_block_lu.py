"""The structure the GPU's subdomain solve rests on, checked on the oracle's matrices.

Section 3 solves each local problem A_i = R_i A R_i^T exactly; the paper uses a sparse
direct solver.  The GPU instead orders a tile of m_x x m_y unknowns by grid rows
(x fastest).  Then:

* A_i is block tridiagonal: diagonal blocks T_j (tridiagonal, the row's own couplings
  and diagonal), off-diagonal blocks C between consecutive rows that are diagonal and
  the same for every row pair (the vertical coupling of column x depends only on x:
  -1/h^2, or -1/(2 h^2) along a Sommerfeld edge);
* block LU S_0 = T_0, S_j = T_j - C S_{j-1}^{-1} C with explicit inverses W_j = S_j^{-1}
  gives the exact solve in 2 m_y - 1 dense block products: forward g_j = W_j (b_j - C g_{j-1}),
  backward x_j = g_j - W_j C x_{j+1}.

Both are checked here, for interior, edge and corner tiles of MP-1 and MP-2 with a
heterogeneous kappa, against the oracle's sparse direct solve (SuperLU) of the same
A_i.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import DIRICHLET, SOMMERFELD, Decomposition, Problem
from paper_2408_03571_gb300.inputs import kappa_field, random_complex_grid


def block_thomas(T, C, b):
    """Solve with diagonal blocks T[j], diagonal coupling vector C, right-hand side rows b[j]."""
    my = len(T)
    W, g = [], []
    S = T[0]
    for j in range(my):
        if j > 0:
            S = T[j] - (C[:, None] * W[j - 1]) * C[None, :]     # T_j - C S_{j-1}^{-1} C
        W.append(np.linalg.inv(S))
        rhs = b[j] if j == 0 else b[j] - C * g[j - 1]
        g.append(W[j] @ rhs)
    x = [None] * my
    x[my - 1] = g[my - 1]
    for j in range(my - 2, -1, -1):
        x[j] = g[j] - W[j] @ (C * x[j + 1])
    return np.concatenate(x)


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
def test_tiles_are_block_tridiagonal_and_block_lu_is_exact(bc):
    n, ns, ov = 33, 4, 2
    prob = Problem(n, bc, kappa_field(n, 14.0, seed=41))
    A = prob.assemble_fast().tocsr()
    dec = Decomposition(prob, ns, ov)
    v = prob.grid_to_vec(random_complex_grid(n, seed=42))
    for s in dec.subs:                      # corner, edge and interior tiles
        Ai = A[s.idx][:, s.idx].toarray()
        mx, my = s.mx, s.my
        T = [Ai[j * mx:(j + 1) * mx, j * mx:(j + 1) * mx] for j in range(my)]
        C = np.diag(Ai[mx:2 * mx, 0:mx]).copy() if my > 1 else np.zeros(mx)
        for j in range(my):
            for jj in range(my):
                blk = Ai[j * mx:(j + 1) * mx, jj * mx:(jj + 1) * mx]
                if abs(j - jj) > 1:
                    assert not np.any(blk)
                elif abs(j - jj) == 1:
                    assert np.array_equal(blk, np.diag(C))        # diagonal, the same for every pair
            assert np.count_nonzero(np.triu(T[j], 2)) == 0 and np.count_nonzero(np.tril(T[j], -2)) == 0
        assert np.all(C != 0)
        b = v[s.idx]
        x = block_thomas(T, C, b.reshape(my, mx))
        ref = spla.splu(A[s.idx][:, s.idx].tocsc()).solve(b)
        assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref)


def block_thomas_c64(T, C, b):
    """The complex64 form: blocks W_j = S_j^{-1} formed in FP64 and rounded to complex64,
    products and the right-hand side in complex64."""
    my = len(T)
    W, S = [], T[0]
    for j in range(my):
        if j > 0:
            S = T[j] - (C[:, None] * W[j - 1]) * C[None, :]
        W.append(np.linalg.inv(S))
    W32 = [w.astype(np.complex64) for w in W]
    C32 = C.real.astype(np.float32)
    b32 = b.astype(np.complex64)
    g = []
    for j in range(my):
        g.append(W32[j] @ (b32[j] if j == 0 else b32[j] - C32 * g[j - 1]))
    x = [None] * my
    x[my - 1] = g[my - 1]
    for j in range(my - 2, -1, -1):
        x[j] = g[j] - W32[j] @ (C32 * x[j + 1])
    return np.concatenate(x).astype(np.complex128)


@pytest.mark.parametrize("bc,n,ns,k,bound", [(DIRICHLET, 129, 2, 40.0, 1e-4), (DIRICHLET, 65, 4, 20.0, 1e-5),
                                            (SOMMERFELD, 65, 4, 20.0, 1e-6)])
def test_complex64_tile_solve_error(bc, n, ns, k, bound):
    """The mixed path's subdomain solve is the same block LU in complex64.  Its relative
    error against the exact local solve is what the mixed-precision parity bars allow
    for (1e-4 on a preconditioner apply): measured 5e-5 at worst (MP-1, n = 129, 2 x 2
    subdomains, k = 40: local Dirichlet problems close to resonance), 3e-6 for MP-1 with
    4 x 4 subdomains at n = 65, 2e-7 on MP-2 boundary tiles.  It stays above FP64
    rounding (the test would not see a path that silently ran in FP64)."""
    prob = Problem(n, bc, k * k)
    A = prob.assemble_fast().tocsr()
    dec = Decomposition(prob, ns, 2)
    v = prob.grid_to_vec(random_complex_grid(n, seed=3))
    worst = 0.0
    for s in dec.subs[:3]:
        Ai = A[s.idx][:, s.idx].toarray()
        mx, my = s.mx, s.my
        T = [Ai[j * mx:(j + 1) * mx, j * mx:(j + 1) * mx] for j in range(my)]
        C = np.diag(Ai[mx:2 * mx, 0:mx]).copy()
        x = block_thomas_c64(T, C, v[s.idx].reshape(my, mx))
        ref = spla.splu(A[s.idx][:, s.idx].tocsc()).solve(v[s.idx])
        worst = max(worst, np.linalg.norm(x - ref) / np.linalg.norm(ref))
    assert 1e-9 < worst <= bound
