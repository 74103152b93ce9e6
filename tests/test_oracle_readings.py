"""Pins for the oracle's alternative readings of the paper (the choices the
paper leaves open, kept selectable to explain the table differences):

* D_i = 1/multiplicity (Section 3 asks only for sum_i R_i^T D_i R_i = I): the
  identity holds, and SAS2 / SHS2 with those D_i equal the dense formulas;
* rectangular subdomain grids (ns_x != ns_y) tile the unknowns;
* B_2 for H = 2^m h as Eq. (7) composed m times: identical to the spline reading
  at m = 1 (Eq. (7)'s printed weights), a partition of unity in the interior, and
  the m = 2 row equals the convolution of Eq. (7)'s stencil with its own upsampled
  copy (computed independently with numpy.convolve);
* left-preconditioned GMRES (Section 5 does not fix the side): each step's
  preconditioned residual is the least-squares minimum over the Krylov space of
  M^{-1} A (brute force), and an exact preconditioner converges in one step.
"""
import numpy as np
import pytest

from oracle import (AS1, B2, DIRICHLET, SAS2, SHS2, SOMMERFELD, CoarseSpace, Decomposition, Problem,
                    Schwarz, basis_1d, gmres)
from paper_2408_03571_gb300.inputs import kappa_field, point_source, random_complex_grid


def _dense_R(idx, N):
    R = np.zeros((len(idx), N))
    R[np.arange(len(idx)), idx] = 1.0
    return R


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
@pytest.mark.parametrize("ns,ov", [((2, 4), 1), ((4, 2), 2), (4, 2), ((1, 2), 0)])
@pytest.mark.parametrize("scaling", ["owner", "multiplicity"])
def test_partition_identity_any_scaling_and_grid(bc, ns, ov, scaling):
    prob = Problem(17, bc, 10.0)
    dec = Decomposition(prob, ns, ov, scaling)
    S = np.zeros((prob.N, prob.N))
    for s in dec.subs:
        R = _dense_R(s.idx, prob.N)
        S += R.T @ np.diag(s.d) @ R
    assert np.allclose(S, np.eye(prob.N), atol=1e-14)
    nsx, nsy = (ns, ns) if np.isscalar(ns) else ns
    assert len(dec.subs) == nsx * nsy


@pytest.mark.parametrize("kind", [SAS2, SHS2])
def test_multiplicity_scaling_dense_formula(kind):
    n, ns, ov, p = 17, 2, 2, 4
    prob = Problem(n, SOMMERFELD, kappa_field(n, 9.0, seed=3))
    A = prob.assemble()
    M = Schwarz(prob, A, ns, ov, kind, B2, p, scaling="multiplicity")
    Ad = A.toarray()
    N = prob.N
    mult = np.zeros(N)
    for s in M.dec.subs:
        mult[s.idx] += 1
    loc_w = np.zeros((N, N), dtype=complex)
    for s in M.dec.subs:
        R = _dense_R(s.idx, N)
        loc_w += R.T @ np.diag(1.0 / mult[s.idx]) @ np.linalg.inv(R @ Ad @ R.T) @ R
    R0 = CoarseSpace(prob, B2, p).R0.toarray()
    Q = R0.T @ np.linalg.inv(R0 @ Ad @ R0.T) @ R0
    Minv = Q + loc_w if kind == SAS2 else Q + loc_w @ (np.eye(N) - Ad @ Q)
    v = prob.grid_to_vec(random_complex_grid(n, seed=6))
    assert np.allclose(M.apply(v), Minv @ v, rtol=1e-10, atol=1e-12 * np.abs(Minv @ v).max())


def test_composed_b2_equals_eq7_at_2h_and_its_convolution_at_4h():
    for n in (9, 17, 33):
        assert np.array_equal(basis_1d(B2, n, 2, True, "composed"), basis_1d(B2, n, 2, True, "spline"))
    W = basis_1d(B2, 65, 4, True, "composed")
    st = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 8.0
    up = np.zeros(9)
    up[::2] = st                               # the level-2 stencil on the fine grid (spacing 2)
    ref = np.convolve(up, st)                  # 13 weights, centred on the coarse node
    I = 8                                      # an interior coarse node (fine node 32)
    assert np.allclose(W[I, 4 * I - 6:4 * I + 7], ref, atol=0)
    assert np.all(W[I, :4 * I - 6] == 0) and np.all(W[I, 4 * I + 7:] == 0)
    # partition of unity away from the boundary, for p = 4, 8
    for p in (4, 8):
        Wp = basis_1d(B2, 129, p, True, "composed")
        assert np.allclose(Wp.sum(axis=0)[2 * p:-2 * p], 1.0, atol=1e-14)


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
def test_left_gmres_minimal_preconditioned_residual_bruteforce(bc):
    n = 17
    prob = Problem(n, bc, 150.0)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, 2, 1, SAS2, B2, 4)
    f = prob.grid_to_vec(point_source(n))
    Mf = M.apply(f)
    K = [Mf]
    for m in range(1, 8):
        r = gmres(lambda x: A @ x, M.apply, f, 1e-30, m, side="left")
        B = np.array([M.apply(A @ k) for k in K]).T        # columns M^{-1} A K_m
        y, *_ = np.linalg.lstsq(B, Mf, rcond=None)
        best = np.linalg.norm(Mf - B @ y) / np.linalg.norm(Mf)
        assert abs(r.resid_hist[-1] - best) <= 1e-9 * max(best, 1e-300) + 1e-13
        K.append(M.apply(A @ K[-1]))


def test_left_gmres_exact_preconditioner_one_step():
    n = 17
    prob = Problem(n, SOMMERFELD, 60.0)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, 1, 0, AS1, None)
    r = gmres(lambda x: A @ x, M.apply, prob.grid_to_vec(point_source(n)), 1e-10, 10, side="left")
    assert r.iterations == 1 and r.converged and r.relres_true < 1e-12
