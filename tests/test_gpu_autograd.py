"""Differentiable solve (adjoint + kappa gradient) through torch.autograd (needs a GB300).

* small grids: the autograd gradient equals the oracle's adjoint gradient
  (oracle dense/sparse solves, same loss), and dL/df equals the oracle's
  adjoint solution;
* the heterogeneous MP-2 workload at n = 1025 (kappa = (100 (1 + 0.2 g))^2, g a
  seeded sum of 16 Gaussian bumps, 64 receivers, target from a perturbed
  field): the gradient matches central finite differences of the loss at 16
  seeded nodes, each difference from two solves at tolerance 1e-10.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")

from oracle import DIRICHLET, SOMMERFELD, Problem  # noqa: E402
from oracle import adjoint as oadj  # noqa: E402
from paper_2408_03571_gb300.inputs import distinct_interior_nodes, kappa_field, point_source  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03571_gb300 import build
    build.build()
    from paper_2408_03571_gb300 import autograd, hzs
    return hzs, autograd


def _loss(u, ut, rec_i, rec_j):
    d = u[rec_j, rec_i] - ut[rec_j, rec_i]
    return 0.5 * (d.abs() ** 2).sum()


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
@pytest.mark.parametrize("prec", [0, 1])
def test_gradient_matches_oracle_adjoint(mods, bc, prec):
    hzs, ag = mods
    n = 65
    kap = kappa_field(n, 18.0, seed=31)
    kap_t = kappa_field(n, 18.0, seed=31, perturb_seed=32)
    f = point_source(n)
    nodes = distinct_interior_nodes(n, 12, seed=33)
    ri = torch.tensor([a for a, _ in nodes], device="cuda")
    rj = torch.tensor([b for _, b in nodes], device="cuda")
    cfg = ag.SolverConfig(bc=0 if bc == DIRICHLET else 1, nsub=4, overlap=2, coarse_ratio=8, precision=prec,
                          tol=1e-11, maxit=400)
    kt = torch.from_numpy(kap).cuda().requires_grad_(True)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    with torch.no_grad():
        ut = ag.solve(torch.from_numpy(kap_t).cuda(), torch.from_numpy(f).cuda(), cfg)
    u = ag.solve(kt, ft, cfg)
    L = _loss(u, ut, ri, rj)
    L.backward()
    # oracle: direct solves and its adjoint gradient for the same loss
    prob = Problem(n, bc, kap)
    A = prob.assemble_fast().tocsc()
    lu = spla.splu(A)
    u_o = lu.solve(prob.grid_to_vec(f))
    ut_o = spla.splu(Problem(n, bc, kap_t).assemble_fast().tocsc()).solve(prob.grid_to_vec(f))
    rec = np.array([prob.index(i, j) for i, j in nodes])
    g = oadj.misfit_residual(u_o, ut_o, rec)
    lam = np.conj(lu.solve(np.conj(g)))                   # conj(A) lam = g
    grad_o = oadj.kappa_gradient(prob.dA_dkappa(), u_o, lam)
    grad = prob.grid_to_vec(kt.grad.cpu().numpy())
    assert np.linalg.norm(grad - grad_o) <= 1e-6 * np.linalg.norm(grad_o)
    gf = prob.grid_to_vec(ft.grad.cpu().numpy())
    assert np.linalg.norm(gf - lam) <= 1e-6 * np.linalg.norm(lam)


def test_gradient_matches_finite_differences_full_size(mods):
    """MP-2, n = 1025, heterogeneous kappa around k = 100, B_2 with H = 1/32."""
    hzs, ag = mods
    n = 1025
    kap = kappa_field(n, 100.0, seed=2001)
    kap_t = kappa_field(n, 100.0, seed=2001, perturb_seed=2002)
    f = torch.from_numpy(point_source(n)).cuda()
    rec = distinct_interior_nodes(n, 64, seed=2003)
    ri = torch.tensor([a for a, _ in rec], device="cuda")
    rj = torch.tensor([b for _, b in rec], device="cuda")
    cfg = ag.SolverConfig(bc=hzs.SOMMERFELD, nsub=16, overlap=2, coarse_ratio=32, precision=hzs.MIXED, tol=1e-6,
                          maxit=800)
    fd_cfg = ag.SolverConfig(bc=hzs.SOMMERFELD, nsub=16, overlap=2, coarse_ratio=32, precision=hzs.MIXED, tol=1e-10,
                             maxit=800)
    with torch.no_grad():
        ut = ag.solve(torch.from_numpy(kap_t).cuda(), f, fd_cfg)
    kt = torch.from_numpy(kap).cuda().requires_grad_(True)
    L = _loss(ag.solve(kt, f, cfg), ut, ri, rj)
    L.backward()
    grad = kt.grad.cpu().numpy()
    gmax = np.abs(grad).max()
    assert np.isfinite(grad).all() and gmax > 0
    for (i, j) in distinct_interior_nodes(n, 16, seed=2004):
        eps = 1e-4 * kap[j, i]
        vals = []
        for s in (+1, -1):
            kp = kap.copy()
            kp[j, i] += s * eps
            with torch.no_grad():
                vals.append(_loss(ag.solve(torch.from_numpy(kp).cuda(), f, fd_cfg), ut, ri, rj).item())
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - grad[j, i]) <= 2e-3 * abs(fd) + 2e-3 * gmax, (i, j, fd, grad[j, i], gmax)
