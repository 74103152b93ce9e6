"""Pins for the oracle's multilevel coarse solve (row f3: the exact coarse solve is
what the paper names the bottleneck for large |G_H|, Section 5).

* one coarse subdomain: SHS2 on G_H is A_0^{-1} exactly (Eq. 6 with a single exact
  local solve), so the outer preconditioner equals the exact two-level one;
* several coarse subdomains: the coarse solve equals the dense SHS2 formula on G_H,
  Q_00 + (sum_i R_0i^T D_0i A_0i^{-1} R_0i)(I - A_0 Q_00), built from explicit
  matrices and numpy inverses;
* with inner GMRES to a tight tolerance, flexible GMRES needs the step count of the
  exact coarse solve.
"""
import numpy as np
import pytest

from oracle import B2, DIRICHLET, SHS2, SOMMERFELD, CoarseSpace, Problem, Schwarz, gmres
from oracle.schwarz import MultilevelCoarseSolver
from paper_2408_03571_gb300.inputs import point_source, random_complex_grid


def _dense_R(idx, N):
    R = np.zeros((len(idx), N))
    R[np.arange(len(idx)), idx] = 1.0
    return R


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
def test_one_coarse_subdomain_is_the_exact_coarse_solve(bc):
    n, k = 65, 12.0
    prob = Problem(n, bc, k * k)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, 16, 2, SHS2, B2, 4)
    ml = MultilevelCoarseSolver(prob, M.coarse.cs, M.coarse.A0, 1, 0, 2)
    c = np.random.default_rng(1).standard_normal(M.coarse.A0.shape[0]) + 0j
    exact = np.linalg.solve(M.coarse.A0, c)
    assert np.linalg.norm(ml.solve(c) - exact) <= 1e-10 * np.linalg.norm(exact)


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
def test_coarse_solve_equals_dense_shs2_on_the_coarse_grid(bc):
    n, k, p, p0 = 65, 10.0, 4, 2
    prob = Problem(n, bc, k * k)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, 16, 2, SHS2, B2, p)
    A0 = M.coarse.A0
    ml = MultilevelCoarseSolver(prob, M.coarse.cs, A0, 2, 1, p0)
    N0 = A0.shape[0]
    loc = np.zeros((N0, N0), dtype=complex)
    for s in ml.M0.dec.subs:
        R = _dense_R(s.idx, N0)
        loc += R.T @ np.diag(s.d) @ np.linalg.inv(R @ A0 @ R.T) @ R
    R00 = CoarseSpace(ml.prob0, B2, p0).R0.toarray()
    Q00 = R00.T @ np.linalg.inv(R00 @ A0 @ R00.T) @ R00
    M0inv = Q00 + loc @ (np.eye(N0) - A0 @ Q00)
    c = np.random.default_rng(2).standard_normal(N0) + 1j * np.random.default_rng(3).standard_normal(N0)
    assert np.allclose(ml.solve(c), M0inv @ c, rtol=1e-10, atol=1e-12 * np.abs(M0inv @ c).max())


def test_inner_iterations_keep_the_outer_step_count():
    k = 40.0
    n = int(round(k / 0.25)) + 1               # the H = 4h regime: kappa h = 0.25
    prob = Problem(n, SOMMERFELD, k * k)
    A = prob.assemble_fast()
    f = prob.grid_to_vec(point_source(n))
    ref = gmres(lambda x: A @ x, Schwarz(prob, A, (n - 1) // 4, 2, SHS2, B2, 4).apply, f, 1e-7, 100)
    M = Schwarz(prob, A, (n - 1) // 4, 2, SHS2, B2, 4, coarse_solve=dict(ns=5, ov=2, p=2, inner_tol=1e-8))
    r = gmres(lambda x: A @ x, M.apply, f, 1e-7, 100, flexible=True)
    assert r.converged and r.iterations == ref.iterations
    assert max(M.coarse.inner.inner_its) < 40
