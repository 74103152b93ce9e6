"""Batched solves (lockstep right-hand sides; several problems at once), through the C ABI.

* hzs_solve with nrhs > 1 gives, per right-hand side, the same iterations and
  the same solution as solving it alone (the batch only changes how the
  kernels are launched), and every solution has the oracle-matrix residual;
* hzs_solve_batched over problems of different wavenumber and grid size gives
  the same per-problem results as separate calls;
* the batched MP-2 workload of the benchmark (64 point sources at seeded nodes
  for each of (k, n) = (25, 257), (50, 257), (100, 513), (200, 1025), 64-node
  subdomains, B_2 with kH <= 1, tol 1e-6) converges for every right-hand side, and
  matches the oracle's solution on the two n = 257 problems.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import B2, SHS2, SOMMERFELD, Problem, Schwarz, gmres  # noqa: E402
from paper_2408_03571_gb300.inputs import point_source, random_source_nodes  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hzs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03571_gb300 import build
    build.build()
    from paper_2408_03571_gb300 import hzs as mod
    return mod


def sources(n, count, seed):
    return torch.from_numpy(np.stack([point_source(n, nd) for nd in random_source_nodes(n, count, seed)])).cuda()


def residuals(n, k, F, U):
    prob = Problem(n, SOMMERFELD, k * k)
    A = prob.assemble_fast()
    out = []
    for f, u in zip(F.cpu().numpy(), U.cpu().numpy()):
        fv, uv = prob.grid_to_vec(f), prob.grid_to_vec(u)
        out.append(np.linalg.norm(fv - A @ uv) / np.linalg.norm(fv))
    return np.array(out)


@pytest.mark.parametrize("prec", [0, 1])
def test_lockstep_batch_equals_single_solves(hzs, prec):
    n, k = 129, 25.0
    g = hzs.Grid(n, hzs.SOMMERFELD, k=k, nsub=4, overlap=2)
    P = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 16, prec)
    F = sources(n, 8, seed=11)
    U, infos = P.solve(F, tol=1e-8, maxit=300)
    assert len(infos) == 8 and all(i.converged for i in infos)
    for r in range(8):
        u1, i1 = P.solve(F[r].contiguous(), tol=1e-8, maxit=300)
        assert i1[0].iterations == infos[r].iterations
        assert torch.linalg.vector_norm(U[r] - u1).item() <= 1e-12 * torch.linalg.vector_norm(u1).item()
    assert np.all(residuals(n, k, F, U) <= 1.01e-8)


def test_multi_problem_batch_equals_separate_calls(hzs):
    probs, rhs, ks = [], [], []
    for (n, k, ns, p, cnt, seed) in [(65, 10.0, 2, 8, 3, 1), (129, 25.0, 4, 16, 5, 2), (97, 15.0, 3, 8, 2, 3)]:
        g = hzs.Grid(n, hzs.SOMMERFELD, k=k, nsub=ns, overlap=2)
        probs.append(hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, p, hzs.MIXED))
        rhs.append(sources(n, cnt, seed))
        ks.append(k)
    outs, res = hzs.solve_batched(probs, rhs, tol=1e-7, maxit=300)
    for P, F, U, R, k in zip(probs, rhs, outs, res, ks):
        U1, R1 = P.solve(F, tol=1e-7, maxit=300)
        assert [r.iterations for r in R] == [r.iterations for r in R1]
        assert torch.equal(U, U1)
        assert np.all(residuals(P.n, k, F, U) <= 1.01e-7)


# The batched MP-2 set of the benchmark: (k, n, subdomains per axis, H/h); 64-node
# subdomains, H the largest power-of-two multiple of h with kH <= 1 (Section 5)
BATCHED = ((25.0, 257, 4, 8), (50.0, 257, 4, 4), (100.0, 513, 8, 4), (200.0, 1025, 16, 4))


def test_batched_mp2_workload(hzs):
    """64 right-hand sides for each of the four problems, solved concurrently; every one
    converges to its true residual, and on the two n = 257 problems the first right-hand
    side's solution matches the oracle's FP64 GMRES solution."""
    probs, rhs, ks = [], [], []
    for idx, (k, n, nsub, p) in enumerate(BATCHED):
        g = hzs.Grid(n, hzs.SOMMERFELD, k=k, nsub=nsub, overlap=2, stream=torch.cuda.Stream())
        probs.append(hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, p, hzs.MIXED))
        rhs.append(sources(n, 64, seed=1000 + idx))
        ks.append(k)
    torch.cuda.synchronize()
    outs, res = hzs.solve_batched(probs, rhs, tol=1e-6, maxit=100)
    torch.cuda.synchronize()
    for P, F, U, R, k in zip(probs, rhs, outs, res, ks):
        assert all(r.converged for r in R)
        assert np.all(residuals(P.n, k, F, U) <= 1.01e-6)
    for (k, n, nsub, p), F, U in list(zip(BATCHED, rhs, outs))[:2]:
        prob = Problem(n, SOMMERFELD, k * k)
        A = prob.assemble_fast()
        M = Schwarz(prob, A, nsub, 2, SHS2, B2, p)
        f = prob.grid_to_vec(F[0].cpu().numpy())
        ref = gmres(lambda x: A @ x, M.apply, f, 1e-6, 300)
        u = prob.grid_to_vec(U[0].cpu().numpy())
        assert ref.converged
        assert np.linalg.norm(u - ref.x) <= 1e-5 * np.linalg.norm(ref.x)
