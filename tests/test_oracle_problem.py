"""Pins for the oracle's discrete model problems (Section 2).

* assembly row-by-row == vectorised assembly (exactly);
* A = A^T for MP-1 and MP-2, A real for MP-1, A != A^H for MP-2 (Section 2);
* interior row sums are -kappa (second-order 5-point stencil);
* MP-1 solution == the closed-form discrete sine-series solution;
* MP-2 boundary rows are consistent with the Sommerfeld condition of Eq. (2):
  applied to outgoing waves they reproduce -Laplace(u) - k^2 u with an error
  that falls with h (a wrong sign or scaling of the boundary term does not);
* MP-2 solution == dense LU (numpy.linalg.solve).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import DIRICHLET, SOMMERFELD, Problem
from paper_2408_03571_gb300.inputs import kappa_field, point_source


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
@pytest.mark.parametrize("n", [5, 9, 17])
@pytest.mark.parametrize("field", [False, True])
def test_assembly_paths_agree(bc, n, field):
    kap = kappa_field(n, 7.0, seed=3) if field else 49.0
    p = Problem(n, bc, kap)
    A1 = p.assemble().toarray()
    A2 = p.assemble_fast().toarray()
    assert np.array_equal(A1, A2)


@pytest.mark.parametrize("n", [9, 17])
def test_symmetry_and_realness(n):
    for bc in (DIRICHLET, SOMMERFELD):
        A = Problem(n, bc, kappa_field(n, 10.0, seed=5)).assemble().toarray()
        assert np.array_equal(A, A.T)
    A1 = Problem(n, DIRICHLET, 100.0).assemble().toarray()
    assert np.all(A1.imag == 0)
    A2 = Problem(n, SOMMERFELD, 100.0).assemble().toarray()
    assert not np.allclose(A2, A2.conj().T)


def test_interior_row_sums():
    n, kap = 17, 37.5
    p = Problem(n, SOMMERFELD, kap)
    A = p.assemble().toarray()
    for j in range(1, n - 1):
        for i in range(1, n - 1):
            assert abs(A[p.index(i, j)].sum() - (-kap)) < 1e-9 * (n - 1) ** 2


def dst_solution(n, k):
    """Closed-form discrete MP-1 solution for the centre source 1/h^2 (sine series)."""
    N = n - 1
    h = 1.0 / N
    c = N // 2
    idx = np.arange(1, N)
    modes = np.arange(1, N)
    S = np.sqrt(2.0 / N) * np.sin(np.pi * np.outer(modes, idx) / N)   # S[p, i]
    lam1 = (4.0 / h**2) * np.sin(modes * np.pi * h / 2) ** 2
    lam = lam1[:, None] + lam1[None, :] - k * k                         # [q, p]
    coef = np.outer(S[:, c - 1], S[:, c - 1]) / (h * h * lam)            # [q, p]
    return S.T @ coef @ S                                                # [j, i] over interior


@pytest.mark.parametrize("n,k", [(9, 5.0), (17, 13.0), (33, 20.0), (65, 20.0)])
def test_mp1_matches_sine_series(n, k):
    p = Problem(n, DIRICHLET, k * k)
    A = p.assemble_fast().tocsc()
    f = p.grid_to_vec(point_source(n))
    u = spla.splu(A).solve(f)
    exact = dst_solution(n, k).ravel()
    assert np.linalg.norm(u - exact) <= 1e-10 * np.linalg.norm(exact)


def test_mp2_matches_dense_solve():
    n = 17
    p = Problem(n, SOMMERFELD, kappa_field(n, 12.0, seed=11))
    A = p.assemble().toarray()
    f = p.grid_to_vec(point_source(n))
    u = spla.splu(p.assemble_fast().tocsc()).solve(f)
    assert np.allclose(u, np.linalg.solve(A, f), rtol=1e-11, atol=0)


def _boundary_row_error(n, k, which):
    p = Problem(n, SOMMERFELD, k * k)
    A = p.assemble_fast()
    x = np.linspace(0.0, 1.0, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    c = n // 3
    if which == "right":      # outgoing through x = 1, du/dx = i k u there
        u = np.exp(1j * k * X) * np.cos(np.pi * Y); node = (n - 1, c); scale = 2.0
        rhs = np.pi**2 * u
    elif which == "left":     # outgoing through x = 0, -du/dx = i k u there
        u = np.exp(-1j * k * X) * np.cos(np.pi * Y); node = (0, c); scale = 2.0
        rhs = np.pi**2 * u
    elif which == "bottom":
        u = np.exp(-1j * k * Y) * np.cos(np.pi * X); node = (c, 0); scale = 2.0
        rhs = np.pi**2 * u
    elif which == "top":
        u = np.exp(1j * k * Y) * np.cos(np.pi * X); node = (c, n - 1); scale = 2.0
        rhs = np.pi**2 * u
    elif which == "corner":   # outgoing through x = 1 and y = 1
        u = np.exp(1j * k * (X + Y)); node = (n - 1, n - 1); scale = 4.0
        rhs = k * k * u
    else:  # corner at the origin
        u = np.exp(-1j * k * (X + Y)); node = (0, 0); scale = 4.0
        rhs = k * k * u
    Au = A @ p.grid_to_vec(u)
    i, j = node
    return abs(scale * Au[p.index(i, j)] - rhs[j, i])


@pytest.mark.parametrize("which", ["right", "left", "bottom", "top", "corner", "corner0"])
def test_sommerfeld_rows_consistent(which):
    k = 3.0
    e = [_boundary_row_error(n, k, which) for n in (33, 65, 129, 257)]
    # consistent (first order at the boundary): error shrinks about 2x per halving of h
    for a, b in zip(e, e[1:]):
        assert b < 0.65 * a
    assert e[-1] < 0.5


def test_dA_dkappa_matches_difference():
    n = 9
    kap = kappa_field(n, 6.0, seed=2)
    p = Problem(n, SOMMERFELD, kap)
    d = p.dA_dkappa()
    eps = 1e-6
    for (i, j) in [(0, 0), (0, 4), (4, 4), (8, 3)]:
        kp = kap.copy(); kp[j, i] += eps
        km = kap.copy(); km[j, i] -= eps
        Ap = Problem(n, SOMMERFELD, kp).assemble().toarray()
        Am = Problem(n, SOMMERFELD, km).assemble().toarray()
        q = p.index(i, j)
        fd = (Ap - Am) / (2 * eps)
        assert abs(fd[q, q] - d[q]) < 1e-6
        fd[q, q] = 0
        assert np.max(np.abs(fd)) < 1e-6   # only the node's own diagonal moves
