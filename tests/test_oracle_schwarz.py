"""Pins for the oracle's Schwarz preconditioners and GMRES (Sections 3 and 5).

* sum_i R_i^T D_i R_i = I (Section 3) and each node lies in at most 4
  subdomains at the largest overlap the paper's experiments use;
* a subdomain is its owned piece grown by `overlap` layers of grid nodes
  (brute-force dilation on the grid), and the owned pieces tile the unknowns;
* AS1, AS2 (Eq. 4), SAS2 (Eq. 5) and SHS2 (Eq. 6) equal the dense formulas
  built from explicit 0/1 matrices and numpy inverses;
* coarse-correction algebra: Q A Q = Q, R_0 (I - A Q) = 0, Q unchanged when
  R_0 is scaled;
* one subdomain => AS1 = A^{-1} => GMRES converges in one step;
* GMRES: each step's residual equals the minimum over the Krylov space found
  by brute-force least squares; Givens rotations zero the subdiagonal;
  flexible GMRES with a fixed preconditioner matches GMRES;
* adjoint gradient == central finite differences of the loss.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import (AS1, AS2, B2, C64, DIRICHLET, P1, SAS2, SHS2, SOMMERFELD, CoarseSpace,
                    Decomposition, Problem, Schwarz, givens, gmres)
from oracle import adjoint
from paper_2408_03571_gb300.inputs import (distinct_interior_nodes, kappa_field, point_source,
                                           random_complex_grid)


def _dense_R(idx, N):
    R = np.zeros((len(idx), N))
    R[np.arange(len(idx)), idx] = 1.0
    return R


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
@pytest.mark.parametrize("ns,ov", [(2, 0), (2, 2), (4, 1), (4, 2), (3, 1)])
def test_partition_identity(bc, ns, ov):
    n = 25 if ns == 3 else 17
    prob = Problem(n, bc, 10.0)
    dec = Decomposition(prob, ns, ov)
    S = np.zeros((prob.N, prob.N))
    mult = np.zeros(prob.N)
    for s in dec.subs:
        R = _dense_R(s.idx, prob.N)
        S += R.T @ np.diag(s.d) @ R
        mult[s.idx] += 1
    assert np.array_equal(S, np.eye(prob.N))
    w = (n - 1) // ns
    if 2 * ov <= w:
        assert mult.max() <= 4


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
@pytest.mark.parametrize("ns,ov", [(2, 1), (4, 2), (3, 3), (4, 0)])
def test_overlap_is_layers_of_nodes_on_every_side(bc, ns, ov):
    """Section 3 extends each nonoverlapping piece by layers of grid nodes: ov rounds of
    adding every unknown adjacent (including diagonally) to the current node set, found
    here by brute-force dilation of the owned nodes on the grid."""
    n = 25
    prob = Problem(n, bc, 10.0)
    dec = Decomposition(prob, ns, ov)
    unknown = np.zeros((n, n), dtype=bool)
    unknown[prob.lo:prob.hi + 1, prob.lo:prob.hi + 1] = True
    owner_count = np.zeros((n, n), dtype=int)
    for s in dec.subs:
        owned = np.zeros((n, n), dtype=bool)               # [j, i]
        for q, dq in zip(s.idx, s.d):
            if dq:
                owned[prob.lo + q // prob.m, prob.lo + q % prob.m] = True
        owner_count += owned
        grown = owned.copy()
        for _ in range(ov):
            nxt = grown.copy()
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    sh = np.zeros_like(grown)
                    sh[max(dj, 0):n + min(dj, 0), max(di, 0):n + min(di, 0)] = \
                        grown[max(-dj, 0):n + min(-dj, 0), max(-di, 0):n + min(-di, 0)]
                    nxt |= sh
            grown = nxt & unknown
        member = np.zeros((n, n), dtype=bool)
        for q in s.idx:
            member[prob.lo + q // prob.m, prob.lo + q % prob.m] = True
        assert np.array_equal(member, grown)
    # the owned pieces tile the unknowns (a nonoverlapping decomposition)
    assert np.array_equal(owner_count, unknown.astype(int))


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
@pytest.mark.parametrize("kind", [AS1, AS2, SAS2, SHS2])
@pytest.mark.parametrize("coarse", [P1, B2])
def test_preconditioner_dense_formula(bc, kind, coarse):
    if kind == AS1 and coarse == P1:
        pytest.skip("AS1 has no coarse space")
    n, ns, ov, p = 17, 2, 2, 4
    prob = Problem(n, bc, kappa_field(n, 9.0, seed=1))
    A = prob.assemble()
    M = Schwarz(prob, A, ns, ov, kind, coarse if kind != AS1 else None, p)
    Ad = A.toarray()
    N = prob.N
    loc_w = np.zeros((N, N), dtype=complex)
    loc = np.zeros((N, N), dtype=complex)
    for s in M.dec.subs:
        R = _dense_R(s.idx, N)
        Ai_inv = np.linalg.inv(R @ Ad @ R.T)
        loc += R.T @ Ai_inv @ R
        loc_w += R.T @ np.diag(s.d) @ Ai_inv @ R
    if kind == AS1:
        Minv = loc
    else:
        R0 = CoarseSpace(prob, coarse, p).R0.toarray()
        Q = R0.T @ np.linalg.inv(R0 @ Ad @ R0.T) @ R0
        Minv = {AS2: Q + loc, SAS2: Q + loc_w,
                SHS2: Q + loc_w @ (np.eye(N) - Ad @ Q)}[kind]
    v = prob.grid_to_vec(random_complex_grid(n, seed=4))
    z = M.apply(v)
    assert np.allclose(z, Minv @ v, rtol=1e-10, atol=1e-12 * np.abs(Minv @ v).max())


def test_coarse_correction_algebra():
    n, p = 33, 4
    prob = Problem(n, SOMMERFELD, 150.0)
    A = prob.assemble_fast()
    Ad = A.toarray()
    R0 = CoarseSpace(prob, B2, p).R0.toarray()
    Q = R0.T @ np.linalg.solve(R0 @ Ad @ R0.T, R0)
    assert np.allclose(Q @ Ad @ Q, Q, atol=1e-10 * np.abs(Q).max())
    P0 = np.eye(prob.N) - Ad @ Q
    assert np.allclose(R0 @ P0, 0, atol=1e-9)
    Q3 = (3 * R0).T @ np.linalg.solve((3 * R0) @ Ad @ (3 * R0).T, 3 * R0)
    assert np.allclose(Q3, Q, atol=1e-12 * np.abs(Q).max())


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
def test_single_subdomain_is_exact(bc):
    n = 17
    prob = Problem(n, bc, 60.0)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, 1, 0, AS1, None)
    f = prob.grid_to_vec(point_source(n))
    r = gmres(lambda x: A @ x, M.apply, f, 1e-10, 10)
    assert r.iterations == 1 and r.converged
    assert r.relres_true < 1e-12


def test_givens_rotation():
    rng = np.random.default_rng(0)
    for _ in range(20):
        a, b = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        c, s = givens(a, b)
        assert isinstance(c, float)
        assert abs(c * c + abs(s) ** 2 - 1) < 1e-14
        assert abs(-np.conj(s) * a + c * b) < 1e-14 * abs(a)
    assert givens(0.0, 2.0)[0] == 0.0


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
def test_gmres_minimal_residual_bruteforce(bc):
    n = 9
    prob = Problem(n, bc, kappa_field(n, 8.0, seed=7))
    A = prob.assemble().toarray()
    M = Schwarz(prob, prob.assemble(), 2, 1, SAS2, B2, 2)
    f = prob.grid_to_vec(random_complex_grid(n, seed=8))
    res = gmres(lambda x: A @ x, M.apply, f, 1e-13, 30)
    # operator B = A M^{-1}; GMRES step m minimises ||f - B y|| over K_m(B, f)
    Mi = np.column_stack([M.apply(e) for e in np.eye(prob.N)])
    B = A @ Mi
    K = [f]
    for m in range(1, min(len(res.resid_hist), 12) + 1):
        Qm, _ = np.linalg.qr(np.column_stack(K))
        y, *_ = np.linalg.lstsq(B @ Qm, f, rcond=None)
        best = np.linalg.norm(f - B @ Qm @ y) / np.linalg.norm(f)
        # the monomial Krylov basis loses accuracy once the residual is small
        tol = 1e-7 if best > 1e-4 else 1e-3
        assert res.resid_hist[m - 1] == pytest.approx(best, rel=tol)
        K.append(B @ K[-1] / np.linalg.norm(K[-1]))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(res.resid_hist, res.resid_hist[1:]))
    assert np.allclose(res.x, np.linalg.solve(A, f), rtol=1e-9)


def test_flexible_matches_fixed():
    n = 17
    prob = Problem(n, SOMMERFELD, 80.0)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, 2, 2, SHS2, B2, 4)
    f = prob.grid_to_vec(point_source(n))
    r1 = gmres(lambda x: A @ x, M.apply, f, 1e-9, 50)
    r2 = gmres(lambda x: A @ x, M.apply, f, 1e-9, 50, flexible=True)
    assert r1.iterations == r2.iterations
    assert np.allclose(r1.x, r2.x, rtol=1e-8)


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
def test_adjoint_gradient_vs_finite_differences(bc):
    n = 17
    kap = kappa_field(n, 11.0, seed=21)
    kap_t = kappa_field(n, 11.0, seed=21, perturb_seed=22)
    f = point_source(n)
    rec_nodes = distinct_interior_nodes(n, 8, seed=23)

    def solve(kk):
        pr = Problem(n, bc, kk)
        return pr, spla.splu(pr.assemble_fast().tocsc()).solve(pr.grid_to_vec(f))

    prob, u = solve(kap)
    _, ut = solve(kap_t)
    rec = np.array([prob.index(i, j) for i, j in rec_nodes])
    g = adjoint.misfit_residual(u, ut, rec)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, 2, 2, SHS2, B2, 4)
    lam, res = adjoint.adjoint_solve(A, M.apply, g, 1e-13, 200)
    assert res.converged
    lam_dense = np.linalg.solve(np.conj(A.toarray()), g)
    assert np.allclose(lam, lam_dense, rtol=1e-9, atol=1e-12 * np.abs(lam_dense).max())
    grad = adjoint.kappa_gradient(prob.dA_dkappa(), u, lam)
    for (i, j) in distinct_interior_nodes(n, 5, seed=24, margin=0) + [(0, 0), (0, 5)]:
        if not prob.is_unknown(i, j):
            continue
        eps = 1e-5 * kap[j, i]
        kp = kap.copy(); kp[j, i] += eps
        km = kap.copy(); km[j, i] -= eps
        Lp = adjoint.loss(solve(kp)[1], ut, rec)
        Lm = adjoint.loss(solve(km)[1], ut, rec)
        fd = (Lp - Lm) / (2 * eps)
        q = prob.index(i, j)
        assert grad[q] == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.abs(grad).max())


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
@pytest.mark.parametrize("kind", [AS1, AS2, SAS2, SHS2])
def test_complex64_preconditioner_is_the_same_operator_rounded(bc, kind):
    """The complex64 mode applies the same M^{-1} as the dense FP64 formula up to
    complex64 rounding (amplified by the condition of the local and coarse
    matrices: 1e-4 relative), is really computed in complex64 (differs from the FP64
    apply by more than FP64 rounding would), and returns complex64 values widened
    exactly to complex128."""
    n, ns, ov, p = 33, 2, 2, 4
    prob = Problem(n, bc, kappa_field(n, 30.0, seed=2))
    A = prob.assemble()
    coarse = None if kind == AS1 else B2
    M64 = Schwarz(prob, A, ns, ov, kind, coarse, p)
    M32 = Schwarz(prob, A, ns, ov, kind, coarse, p, precision=C64)
    Ad = A.toarray()
    N = prob.N
    loc_w = np.zeros((N, N), dtype=complex)
    loc = np.zeros((N, N), dtype=complex)
    for s in M64.dec.subs:
        R = _dense_R(s.idx, N)
        Ai_inv = np.linalg.inv(R @ Ad @ R.T)
        loc += R.T @ Ai_inv @ R
        loc_w += R.T @ np.diag(s.d) @ Ai_inv @ R
    if kind == AS1:
        Minv = loc
    else:
        R0 = CoarseSpace(prob, coarse, p).R0.toarray()
        Q = R0.T @ np.linalg.inv(R0 @ Ad @ R0.T) @ R0
        Minv = {AS2: Q + loc, SAS2: Q + loc_w, SHS2: Q + loc_w @ (np.eye(N) - Ad @ Q)}[kind]
    v = prob.grid_to_vec(random_complex_grid(n, seed=8))
    ref = Minv @ v
    z32 = M32.apply(v)
    err = np.linalg.norm(z32 - ref) / np.linalg.norm(ref)
    assert 1e-9 < err < 1e-4
    assert np.linalg.norm(M64.apply(v) - ref) / np.linalg.norm(ref) < 1e-12
    assert z32.dtype == np.complex128
    assert np.array_equal(z32.astype(np.complex64).astype(np.complex128), z32)


def test_complex64_deflation_annihilates_the_coarse_residual():
    """SHS2 in complex64: the deflated residual w = v - A Q v has R_0 w = 0 up to
    complex64 rounding (R_0 (I - A Q) = 0, Eq. (6)), i.e. the coarse correction
    and the deflation use the same transfers."""
    n, p = 65, 8
    prob = Problem(n, DIRICHLET, 400.0)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, 4, 2, SHS2, B2, p, precision=C64)
    v = prob.grid_to_vec(random_complex_grid(n, seed=5)).astype(np.complex64)
    w = v - M.Ap @ M.apply_Q(v)
    R0 = CoarseSpace(prob, B2, p).R0
    assert np.linalg.norm(R0 @ w) / np.linalg.norm(R0 @ v) < 2e-5


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
def test_complex64_flexible_gmres_reaches_tol(bc):
    """Flexible GMRES in FP64 around the complex64 preconditioner reaches the
    tolerance in its true residual, in a few more steps than around the FP64 one
    (a perturbed preconditioner), and its solution matches the FP64 solve to 1e-5."""
    n, k = 65, 20.0
    prob = Problem(n, bc, k * k)
    A = prob.assemble_fast()
    f = prob.grid_to_vec(point_source(n))
    r64 = gmres(lambda x: A @ x, Schwarz(prob, A, 4, 2, SHS2, B2, 8).apply, f, 1e-7, 200, True)
    r32 = gmres(lambda x: A @ x, Schwarz(prob, A, 4, 2, SHS2, B2, 8, precision=C64).apply, f, 1e-7, 200, True)
    assert r32.converged and r32.relres_true <= 1.01e-7
    assert r64.iterations <= r32.iterations <= r64.iterations + 6
    assert np.linalg.norm(r32.x - r64.x) / np.linalg.norm(r64.x) < 1e-5
