"""Pins for the oracle's coarse spaces (Section 4).

* B_2 at H = 2h reproduces the printed weights (1, 4, 6, 4, 1)/8 of Eq. (7)
  (golden fixture tests/golden/b2_weights_h2.txt);
* the cardinal quadratic B-spline: known values, symmetry, unit integral,
  C^1 joins; partition of unity of the shifted family for every p;
* P_1 hats are interpolatory (phi_I(X_J) = delta_IJ) and sum to one;
* R_0 equals the brute-force tensor product phi_I(x_i) phi_J(y_j);
* A_0 has the same size for P_1 and B_2; its interior stencil has 9 points
  for P_1 and 25 for B_2 (Section 4, "lower sparseness");
* grid and coarse-grid node counts of Tables 1-2 (golden fixture);
* each fine node meets at most 3 consecutive B_2 (2 P_1) functions per axis.
"""
import os

import numpy as np
import pytest

from oracle import B2, DIRICHLET, P1, SOMMERFELD, CoarseSpace, Problem, basis_1d, bspline2

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t) for t in line.split()])
    return rows


def test_b2_weights_h2_match_eq7():
    gold = {off: num / den for off, num, den in _load("b2_weights_h2.txt")}
    n, p = 17, 2
    W = basis_1d(B2, n, p, keep_ends=True)
    # an interior coarse node I sits on fine node 2I
    for I in (2, 3, 5):
        row = W[I]
        for off, val in gold.items():
            assert row[2 * I + off] == pytest.approx(val, abs=1e-15)
        nz = np.nonzero(row)[0]
        assert set(nz - 2 * I) == set(gold)


def test_bspline_closed_form():
    assert bspline2(np.array([0.5, 1.0, 1.5, 2.0, 2.5])) == pytest.approx([1 / 8, 1 / 2, 3 / 4, 1 / 2, 1 / 8])
    t = np.linspace(-1, 4, 5001)
    b = bspline2(t)
    assert np.all(b[(t < 0) | (t > 3)] == 0)
    assert np.allclose(b, bspline2(3 - t))                         # symmetric about 3/2
    tt = np.linspace(0, 3, 300001)
    integral = np.sum(bspline2(tt)) * (tt[1] - tt[0])
    assert integral == pytest.approx(1.0, abs=1e-5)
    e = 1e-7                                                       # C^1 at the knots
    for knot in (1.0, 2.0):
        dl = (bspline2(knot) - bspline2(knot - e)) / e
        dr = (bspline2(knot + e) - bspline2(knot)) / e
        assert dl == pytest.approx(dr, abs=1e-5)


@pytest.mark.parametrize("kind", [B2, P1])
@pytest.mark.parametrize("p", [2, 4, 8, 32])
def test_partition_of_unity(kind, p):
    n = 4 * p * 4 + 1
    W = basis_1d(kind, n, p, keep_ends=True)
    s = W.sum(axis=0)
    # B_2 needs the missing function beyond the boundary within H/2 of each end
    margin = (p // 2 + 1) if kind == B2 else 0
    assert np.allclose(s[margin:n - margin], 1.0, atol=1e-14)


def test_p1_interpolatory():
    n, p = 33, 4
    W = basis_1d(P1, n, p, keep_ends=True)
    nodes = np.arange(0, n, p)
    assert np.allclose(W[:, nodes], np.eye(len(nodes)))


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
@pytest.mark.parametrize("kind", [B2, P1])
def test_R0_is_tensor_product(bc, kind):
    n, p = 17, 4
    prob = Problem(n, bc, 30.0)
    cs = CoarseSpace(prob, kind, p)
    keep = bc == SOMMERFELD
    W = basis_1d(kind, n, p, keep)
    R = cs.R0.toarray()
    for J in range(W.shape[0]):
        for I in range(W.shape[0]):
            row = R[J * W.shape[0] + I]
            for j in range(prob.lo, prob.hi + 1):
                for i in range(prob.lo, prob.hi + 1):
                    assert row[prob.index(i, j)] == W[I, i] * W[J, j]
    nc1 = (n - 1) // p + 1 - (0 if keep else 2)
    assert R.shape == (nc1 * nc1, prob.N)


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
def test_coarse_matrix_size_and_stencil(bc):
    n, p = 65, 8
    prob = Problem(n, bc, 100.0)
    A = prob.assemble_fast()
    A0 = {kind: CoarseSpace(prob, kind, p).galerkin(A) for kind in (P1, B2)}
    assert A0[P1].shape == A0[B2].shape
    nc1 = CoarseSpace(prob, P1, p).nc1
    mid = (nc1 // 2) * nc1 + nc1 // 2
    assert np.count_nonzero(np.abs(A0[P1][mid]) > 1e-12) == 9
    assert np.count_nonzero(np.abs(A0[B2][mid]) > 1e-12) == 25
    assert np.allclose(A0[B2], A0[B2].T)


def test_table_grid_counts():
    for nsub, Gh, GH, inv_h, inv_H, k in _load("grid_counts.txt"):
        n = inv_h + 1
        assert n * n == Gh
        p = inv_h // inv_H
        assert p == 4
        assert ((n - 1) // p + 1) ** 2 == GH                       # coarse nodes incl. boundary
        assert (inv_h // 4) ** 2 == nsub                           # H_sub = 4h
        assert k / inv_h == pytest.approx(0.25)                    # kappa_h = 0.25
        W = basis_1d(B2, n, p, keep_ends=True)
        assert W.shape[0] ** 2 == GH


@pytest.mark.parametrize("p", [2, 3, 4, 8, 16, 32])
def test_each_fine_node_meets_few_coarse_functions(p):
    """Every fine node lies in the support of at most 3 B_2 functions and at most 2 P_1
    hats per axis (B_2 is supported on 3 coarse cells, a hat on 2), and those coarse
    indices are consecutive: per axis a node needs its first coarse index and up to three
    weights, which is how the GPU's restriction and prolongation tables store R_0."""
    n = 8 * p + 1
    for kind, most in ((B2, 3), (P1, 2)):
        W = basis_1d(kind, n, p, keep_ends=True)
        for i in range(n):
            nz = np.nonzero(W[:, i])[0]
            assert 1 <= len(nz) <= most
            assert np.array_equal(nz, np.arange(nz[0], nz[0] + len(nz)))
