"""GPU parity of the selectable readings of the boundary (through the C ABI):

* D_i = 1/multiplicity for SAS2 and SHS2 (hzs_precond_desc.scaling_mode;
  Section 3 only asks for sum_i R_i^T D_i R_i = I): the preconditioner against
  the oracle's (FP64 1e-9, complex64 1e-4), and a solve within one step of the
  oracle's GMRES with the same D_i;
* rectangular subdomain grids (hzs_grid_desc.nsub_y): every preconditioner kind
  against the oracle's with the same ns_x x ns_y decomposition.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import AS1, AS2, B2, DIRICHLET, P1, SAS2, SHS2, SOMMERFELD, Problem, Schwarz, gmres  # noqa: E402
from paper_2408_03571_gb300.inputs import point_source, random_complex_grid  # noqa: E402

pytestmark = pytest.mark.gpu

BC = {DIRICHLET: 0, SOMMERFELD: 1}
KIND = {AS1: 0, AS2: 1, SAS2: 2, SHS2: 3}
COARSE = {None: 0, P1: 1, B2: 2}


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


@pytest.mark.parametrize("prec,bar", [(0, 1e-9), (1, 1e-4)])
@pytest.mark.parametrize("kind", [SAS2, SHS2])
@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
def test_multiplicity_scaling_preconditioner(hzs, bc, kind, prec, bar):
    n, nsub, ov, p, k = 65, 4, 2, 8, 14.0
    prob = Problem(n, bc, k * k)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, nsub, ov, kind, B2, p, scaling="multiplicity")
    g = hzs.Grid(n, BC[bc], k=k, nsub=nsub, overlap=ov)
    P = hzs.Preconditioner(g, KIND[kind], COARSE[B2], p, prec, scaling_mode=hzs.SCALING_MULTIPLICITY)
    v = random_complex_grid(n, seed=9)
    z = P.apply(dev(v)).cpu().numpy()
    ref = prob.vec_to_grid(M.apply(prob.grid_to_vec(v)))
    assert rel(z, ref) < bar


@pytest.mark.parametrize("kind", [SAS2, SHS2])
def test_multiplicity_scaling_solve(hzs, kind):
    n, nsub, ov, p, k = 81, 20, 2, 4, 20.0
    prob = Problem(n, SOMMERFELD, k * k)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, nsub, ov, kind, B2, p, scaling="multiplicity")
    f = point_source(n)
    ref = gmres(lambda x: A @ x, M.apply, prob.grid_to_vec(f), 1e-7, 100)
    g = hzs.Grid(n, 1, k=k, nsub=nsub, overlap=ov)
    P = hzs.Preconditioner(g, KIND[kind], COARSE[B2], p, 0, scaling_mode=hzs.SCALING_MULTIPLICITY)
    u, info = P.solve(dev(f), tol=1e-7, maxit=100)
    assert info[0].converged and abs(info[0].iterations - ref.iterations) <= 1
    assert rel(prob.grid_to_vec(u.cpu().numpy()), ref.x) < 1e-5


@pytest.mark.parametrize("kind,coarse", [(AS1, None), (AS2, P1), (SAS2, B2), (SHS2, B2)])
@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
@pytest.mark.parametrize("nsx,nsy", [(2, 8), (8, 4)])
def test_rectangular_subdomain_grid(hzs, bc, kind, coarse, nsx, nsy):
    n, ov, p, k = 65, 2, 8, 12.0
    prob = Problem(n, bc, k * k)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, (nsx, nsy), ov, kind, coarse, p)
    g = hzs.Grid(n, BC[bc], k=k, nsub=nsx, nsub_y=nsy, overlap=ov)
    P = hzs.Preconditioner(g, KIND[kind], COARSE[coarse], p, 0)
    v = random_complex_grid(n, seed=12)
    z = P.apply(dev(v)).cpu().numpy()
    ref = prob.vec_to_grid(M.apply(prob.grid_to_vec(v)))
    assert rel(z, ref) < 1e-9


def test_bad_readings_rejected(hzs):
    g = hzs.Grid(65, 0, k=10.0, nsub=4, overlap=2)
    with pytest.raises(hzs.HzsError) as e:
        hzs.Preconditioner(g, hzs.SAS2, hzs.COARSE_B2, 8, 0, scaling_mode=7)
    assert e.value.status == hzs.ERR_INVALID_ARG
    with pytest.raises(hzs.HzsError) as e:
        hzs.Grid(65, 0, k=10.0, nsub=4, nsub_y=3, overlap=2)          # 3 does not divide 64
    assert e.value.status == hzs.ERR_INVALID_ARG
