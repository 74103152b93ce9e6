"""The multilevel coarse solve on the GPU (HZS_COARSE_SOLVER_MULTILEVEL) against the
oracle's MultilevelCoarseSolver, through the C ABI.

A_0^{-1} is replaced by one application of SHS2 (Eq. 6) on the coarse grid G_H: coarse
subdomains with exact solves of their blocks of A_0, a B_2 coarse-of-coarse space with
its own exact Galerkin solve (Section 5 names the exact coarse solve as the cost that
grows with |G_H|).  Checked, in the H = 4h setting of the paper's first two tables:

* the preconditioner apply equals the oracle's (FP64 1e-9, complex64 preconditioner
  1e-4), MP-1 and MP-2, SHS2 and AS2;
* with a single coarse subdomain it is the exact coarse solve (the DENSE solver's apply);
* its coarse-of-coarse solve by block LU (above 4096 unknowns) equals the dense one;
* a GMRES solve takes the oracle's step count (+-1) with the same preconditioner and
  reaches the same solution;
* parameters that do not fit the coarse grid are rejected.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import AS2, B2, C64, DIRICHLET, SHS2, SOMMERFELD, Problem, Schwarz, gmres  # noqa: E402
from paper_2408_03571_gb300.inputs import point_source, random_complex_grid  # noqa: E402

pytestmark = pytest.mark.gpu

BC = {DIRICHLET: 0, SOMMERFELD: 1}
KIND = {AS2: 1, SHS2: 3}


@pytest.fixture(scope="module")
def hzs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03571_gb300 import build
    build.build()
    from paper_2408_03571_gb300 import hzs as mod
    return mod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def regime(k):
    """kappa h = 0.25, H_sub = H = 4h, overlap 2 (the paper's first two tables)."""
    n = int(round(k / 0.25)) + 1
    return n, (n - 1) // 4


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
@pytest.mark.parametrize("kind", [SHS2, AS2])
@pytest.mark.parametrize("prec,bar", [(0, 1e-9), (1, 1e-4)])
def test_apply_matches_oracle(hzs, bc, kind, prec, bar):
    k = 40.0
    n, ns = regime(k)
    prob = Problem(n, bc, k * k)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, ns, 2, kind, B2, 4, precision="fp64" if prec == 0 else C64,
                coarse_solve=dict(ns=5, ov=2, p=2))
    g = hzs.Grid(n, BC[bc], k=k, nsub=ns, overlap=2)
    P = hzs.Preconditioner(g, KIND[kind], hzs.COARSE_B2, 4, prec, coarse_solver=hzs.COARSE_SOLVER_MULTILEVEL,
                           ml=(5, 2, 2))
    assert P.info()["coarse_solver"] == hzs.COARSE_SOLVER_MULTILEVEL
    v = random_complex_grid(n, seed=21)
    z = P.apply(dev(v)).cpu().numpy()
    ref = prob.vec_to_grid(M.apply(prob.grid_to_vec(v)))
    assert rel(z, ref) < bar


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
def test_one_coarse_subdomain_is_the_exact_coarse_solve(hzs, bc):
    k = 20.0
    n, ns = regime(k)
    g = hzs.Grid(n, BC[bc], k=k, nsub=ns, overlap=2)
    Pe = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 4, 0, coarse_solver=hzs.COARSE_SOLVER_DENSE)
    Pm = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 4, 0, coarse_solver=hzs.COARSE_SOLVER_MULTILEVEL,
                            ml=(1, 0, 2))
    v = dev(random_complex_grid(n, seed=22))
    ze = Pe.apply(v).cpu().numpy()
    zm = Pm.apply(v).cpu().numpy()
    assert rel(zm, ze) < 1e-9


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
def test_solve_matches_oracle(hzs, bc):
    k = 40.0
    n, ns = regime(k)
    prob = Problem(n, bc, k * k)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, ns, 2, SHS2, B2, 4, coarse_solve=dict(ns=5, ov=2, p=2))
    f = point_source(n)
    ref = gmres(lambda x: A @ x, M.apply, prob.grid_to_vec(f), 1e-7, 100)
    g = hzs.Grid(n, BC[bc], k=k, nsub=ns, overlap=2)
    P = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 4, 0, coarse_solver=hzs.COARSE_SOLVER_MULTILEVEL,
                           ml=(5, 2, 2))
    u, info = P.solve(dev(f), tol=1e-7, maxit=100)
    assert ref.converged and info[0].converged
    assert abs(info[0].iterations - ref.iterations) <= 1
    assert info[0].relres_true <= 1.01e-7
    assert rel(prob.grid_to_vec(u.cpu().numpy()), ref.x) < 1e-5


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
def test_block_coarse_of_coarse_equals_dense(hzs, bc, monkeypatch):
    """Above 4096 coarse-of-coarse unknowns their solve is a block-tridiagonal LU of A_00
    (a band of radius 3, groups of 3 rows); HZS_ML_BLOCK00=1 takes it at a size where
    the dense inverse also runs, and both are the same exact solve."""
    k = 40.0
    n, ns = regime(k)
    g = hzs.Grid(n, BC[bc], k=k, nsub=ns, overlap=2)
    v = dev(random_complex_grid(n, seed=23))
    kw = dict(coarse_solver=hzs.COARSE_SOLVER_MULTILEVEL, ml=(5, 2, 2))
    zd = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 4, 0, **kw).apply(v).cpu().numpy()
    monkeypatch.setenv("HZS_ML_BLOCK00", "1")
    zb = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 4, 0, **kw).apply(v).cpu().numpy()
    assert rel(zb, zd) < 1e-10


def test_bad_parameters_rejected(hzs):
    k = 20.0
    n, ns = regime(k)                      # G_H: 21 coarse nodes per axis (MP-2)
    g = hzs.Grid(n, 1, k=k, nsub=ns, overlap=2)
    for ml in [(3, 1, 2), (5, 3, 2), (5, 1, 3), (5, 1, 1), (0, 0, 2)]:
        with pytest.raises(hzs.HzsError) as e:
            hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 4, 0, coarse_solver=hzs.COARSE_SOLVER_MULTILEVEL, ml=ml)
        assert e.value.status == hzs.ERR_INVALID_ARG
