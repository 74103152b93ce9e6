"""Failure statuses through the C ABI, in forms that fault, trap or hang no GPU.

* HZS_ERR_SINGULAR_LOCAL: a decomposition into one-node subdomains of MP-2 with
  kappa = 4/h^2, so every interior local matrix is the 1 x 1 matrix 4/h^2 - kappa
  = 0 exactly (Section 3's exact local solve has nothing to invert).
* HZS_ERR_SINGULAR_COARSE: MP-1, n = 5, the P_1 coarse space with H = 2h has one
  coarse function r; a kappa field (16 everywhere, 28 at the centre) makes
  A_0 = r^T A r = 0 exactly in binary arithmetic (Eq. 4's coarse matrix is
  singular) while the one local matrix stays regular.
* HZS_ERR_TIMEOUT: the subdomain solve's waits for its factor copies are given a
  limit of zero polls (HZS_STAGE_WAIT_POLLS=0, read at set-up): every block gives up
  at its first wait, records the status, waits with the full limit for the copies
  it started and returns; the solve reports the status and the context stays
  usable (a handle set up afterwards with the default limit solves normally).
Each case checks the status and the message; none plants a fault.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import DIRICHLET, P1, CoarseSpace, Problem  # noqa: E402
from paper_2408_03571_gb300.inputs import point_source  # noqa: E402


def singular_coarse_kappa(n=5):
    kap = np.full((n, n), 16.0)
    kap[n // 2, n // 2] = 28.0
    return kap


def test_singular_coarse_case_is_exactly_singular():
    """CPU check of the case itself: the oracle's A_0 is exactly zero, the local matrix is not singular."""
    prob = Problem(5, DIRICHLET, singular_coarse_kappa())
    A = prob.assemble()
    A0 = CoarseSpace(prob, P1, 2).galerkin(A)
    assert A0.shape == (1, 1) and A0[0, 0] == 0
    assert abs(np.linalg.det(A.toarray())) > 1e3


@pytest.fixture(scope="module")
def hzs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03571_gb300 import build
    build.build()
    from paper_2408_03571_gb300 import hzs as mod
    return mod


@pytest.mark.gpu
def test_singular_local_matrix_reported_at_setup(hzs):
    n = 9                                     # h = 1/8: 4/h^2 = 256 = k^2 for k = 16, exactly
    g = hzs.Grid(n, hzs.SOMMERFELD, k=16.0, nsub=n - 1, overlap=0)
    with pytest.raises(hzs.HzsError) as e:
        hzs.Preconditioner(g, hzs.AS1, hzs.COARSE_NONE, 2, hzs.FP64)
    assert e.value.status == hzs.ERR_SINGULAR_LOCAL
    assert "subdomain" in str(e.value)


@pytest.mark.gpu
def test_singular_coarse_matrix_reported_at_setup(hzs):
    n = 5
    kap = torch.from_numpy(singular_coarse_kappa(n)).cuda()
    g = hzs.Grid(n, hzs.DIRICHLET, kappa=kap, nsub=1, overlap=0)
    with pytest.raises(hzs.HzsError) as e:
        hzs.Preconditioner(g, hzs.SAS2, hzs.COARSE_P1, 2, hzs.FP64)
    assert e.value.status == hzs.ERR_SINGULAR_COARSE
    assert "coarse" in str(e.value)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_stage_wait_timeout_reported_and_context_usable(hzs, prec, monkeypatch):
    n = 65
    f = torch.from_numpy(point_source(n)).cuda()
    g = hzs.Grid(n, hzs.DIRICHLET, k=20.0, nsub=4, overlap=2)
    monkeypatch.setenv("HZS_STAGE_WAIT_POLLS", "0")
    P = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 8, prec)
    monkeypatch.delenv("HZS_STAGE_WAIT_POLLS")
    with pytest.raises(hzs.HzsError) as e:
        P.solve(f, tol=1e-7, maxit=5)
    assert e.value.status == hzs.ERR_TIMEOUT
    P.close()
    torch.cuda.synchronize()                  # the context is intact: no sticky error
    P2 = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 8, prec)
    u, info = P2.solve(f, tol=1e-7, maxit=200)
    assert info[0].converged and info[0].relres_true <= 1.01e-7
