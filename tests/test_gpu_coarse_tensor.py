"""Block coarse solve with many right-hand sides on the tensor cores, through the C ABI.

With more than two right-hand sides the sweeps of the block-tridiagonal coarse solve
A_0^{-1} (Eq. 4) form W_i X for all of them at once, as FP64-accurate digit-slice products
on the tensor cores (bf16 slices of 7 bits, exact FP32 accumulation, sum in FP32
expansions, one rounding to FP64).  Checked here:

* the preconditioner apply of several right-hand sides equals the oracle's (FP64 bar
  1e-9), the dense-inverse coarse solve and the same sweeps on the FP64 pipe
  (HZS_COARSE_TC=0) to 1e-11, MP-1 and MP-2, B_2 and P_1, ragged block sizes;
* at the widest blocks (n = 1025, H = 4h: 257 coarse nodes a row, blocks of 514, K = 1028,
  the limit of exact accumulation) against the FP64-pipe sweeps;
* numbers of right-hand sides that do not fill a 32-column tile (3, 5, 17), and 64 (four
  column tiles);
* a batched GMRES solve takes the same steps and reaches the same solutions as with the
  FP64-pipe sweeps, right-hand sides that converge early included;
* the preconditioner reports which form it built.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import B2, DIRICHLET, P1, SHS2, SOMMERFELD, Problem, Schwarz  # noqa: E402
from paper_2408_03571_gb300.inputs import point_source, random_complex_grid, random_source_nodes  # noqa: E402

pytestmark = pytest.mark.gpu

BC = {DIRICHLET: 0, SOMMERFELD: 1}
COARSE = {P1: 1, B2: 2}
BLOCK, DENSE = 2, 1


@pytest.fixture(scope="module")
def hzs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03571_gb300 import build
    build.build()
    from paper_2408_03571_gb300 import hzs as mod
    return mod


@pytest.fixture
def fp64_sweeps(monkeypatch):
    """Builds preconditioners whose block sweeps stay on the FP64 pipe."""
    def make(fn):
        monkeypatch.setenv("HZS_COARSE_TC", "0")
        try:
            return fn()
        finally:
            monkeypatch.delenv("HZS_COARSE_TC")
    return make


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def batch(n, nrhs, seed):
    return np.stack([random_complex_grid(n, seed=seed + r) for r in range(nrhs)])


@pytest.mark.parametrize("bc", [DIRICHLET, SOMMERFELD])
@pytest.mark.parametrize("coarse", [B2, P1])
def test_many_rhs_apply_vs_oracle(hzs, fp64_sweeps, bc, coarse):
    n, nsub, ov, p, k = 65, 16, 2, 4, 14.0          # H = 4h: ragged last block of one row
    nrhs = 5
    prob = Problem(n, bc, k * k)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, nsub, ov, SHS2, coarse, p)
    V = batch(n, nrhs, 40)
    g = hzs.Grid(n, BC[bc], k=k, nsub=nsub, overlap=ov)
    Pt = hzs.Preconditioner(g, hzs.SHS2, COARSE[coarse], p, 0, True, BLOCK)
    Pf = fp64_sweeps(lambda: hzs.Preconditioner(g, hzs.SHS2, COARSE[coarse], p, 0, True, BLOCK))
    Pd = hzs.Preconditioner(g, hzs.SHS2, COARSE[coarse], p, 0, True, DENSE)
    assert Pt.info()["coarse_tensor_cores"] == 1
    assert Pf.info()["coarse_tensor_cores"] == 0 and Pd.info()["coarse_tensor_cores"] == 0
    zt = Pt.apply(dev(V)).cpu().numpy()
    zf = Pf.apply(dev(V)).cpu().numpy()
    zd = Pd.apply(dev(V)).cpu().numpy()
    for r in range(nrhs):
        ref = prob.vec_to_grid(M.apply(prob.grid_to_vec(V[r])))
        assert rel(zt[r], ref) < 1e-9
        assert rel(zt[r], zd[r]) < 1e-11
        assert rel(zt[r], zf[r]) < 1e-11


@pytest.mark.parametrize("nrhs", [3, 17])
def test_many_rhs_apply_mixed(hzs, fp64_sweeps, nrhs):
    """The complex64 preconditioner: its coarse solve is FP64 either way."""
    n, nsub, ov, p, k = 129, 8, 2, 4, 30.0
    V = batch(n, nrhs, 60)
    g = hzs.Grid(n, 1, k=k, nsub=nsub, overlap=ov)
    Pt = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, p, 1, True, BLOCK)
    Pf = fp64_sweeps(lambda: hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, p, 1, True, BLOCK))
    zt = Pt.apply(dev(V)).cpu().numpy()
    zf = Pf.apply(dev(V)).cpu().numpy()
    for r in range(nrhs):
        assert rel(zt[r], zf[r]) < 1e-6           # complex64 transfers around the same coarse solve


def test_widest_blocks(hzs, fp64_sweeps):
    """n = 1025, H = 4h: blocks of 2 x 257 coarse rows, K = 1028 in the digit products."""
    n, nsub, ov, p, k = 1025, 16, 2, 4, 200.0
    nrhs = 4
    V = batch(n, nrhs, 80)
    g = hzs.Grid(n, 1, k=k, nsub=nsub, overlap=ov)
    Pt = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, p, 0, True, BLOCK)
    assert Pt.info()["coarse_tensor_cores"] == 1 and Pt.info()["coarse_unknowns"] == 257 * 257
    zt = Pt.apply(dev(V)).cpu().numpy()
    Pt.close()
    Pf = fp64_sweeps(lambda: hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, p, 0, True, BLOCK))
    zf = Pf.apply(dev(V)).cpu().numpy()
    for r in range(nrhs):
        assert rel(zt[r], zf[r]) < 1e-11


@pytest.mark.parametrize("prec,nrhs", [(0, 8), (1, 8), (0, 64)])
def test_batched_solve_same_steps(hzs, fp64_sweeps, prec, nrhs):
    """FP64 preconditioner: the same steps; complex64 (whose coarse solution is rounded to
    complex64 after the FP64 solve, so a last-bit difference there can flip a rounding):
    within one step.  64 right-hand sides fill four 32-column tiles."""
    n, nsub, ov, p, k = 257, 4, 2, 4, 50.0
    nodes = random_source_nodes(n, nrhs, 7)
    F = np.stack([point_source(n, nd) for nd in nodes])
    F[5] = point_source(n)                              # the centre source: its own step count
    g = hzs.Grid(n, 1, k=k, nsub=nsub, overlap=ov)
    Pt = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, p, prec, True, BLOCK)
    Pf = fp64_sweeps(lambda: hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, p, prec, True, BLOCK))
    ut, it = Pt.solve(dev(F), tol=1e-8, maxit=100)
    uf, inf = Pf.solve(dev(F), tol=1e-8, maxit=100)
    ut, uf = ut.cpu().numpy(), uf.cpu().numpy()
    assert len({r.iterations for r in inf}) > 1          # the batch really has members that stop early
    for r in range(nrhs):
        assert it[r].converged and inf[r].converged
        assert abs(it[r].iterations - inf[r].iterations) <= (0 if prec == 0 else 1)
        assert it[r].relres_true <= 1.01e-8
        assert rel(ut[r], uf[r]) < (1e-9 if prec == 0 else 1e-6)
