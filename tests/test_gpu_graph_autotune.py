"""Graph-issued Arnoldi steps and the subdomain-solve autotuner, through the C ABI.

* HZS_SOLVE_GRAPH captures the steps in chunks of 8 and replays them: the same
  kernels with the same arguments in the same order as the stream-issued solve,
  so the same step counts, estimates and solutions (to 1e-12 relative) - for
  the FP64 path, both mixed-precision orthogonalisations, a lockstep batch whose
  entries finish at different steps, a solve stopped by maxit inside a chunk,
  the adjoint solve, hzs_solve_batched over two problems on their own streams,
  and a second solve of the same handle (the executable graphs are reused);
* autotune = 2 times the launch shapes of the subdomain solve that fit, reports
  the one it keeps (never slower than the default by its own timing), and the
  tuned preconditioner applies the same z = M^{-1} v as the default one (the
  same tile systems; only the order of a block row's partial sums may change):
  FP64 to 1e-11 and complex64 to 1e-4 relative (a complex64 apply agrees with
  the FP64 one to about 1e-5, so two complex64 summation orders agree within
  that); its solves take the default's step count (within 1 for FP64, 3 for
  the perturbed complex64 preconditioner) and meet tol in the true residual of
  the oracle's matrix; autotune = 1 reuses the choice.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import DIRICHLET, SOMMERFELD, Problem  # noqa: E402
from paper_2408_03571_gb300.inputs import point_source, random_complex_grid, random_source_nodes  # noqa: E402

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


OBC = {0: DIRICHLET, 1: SOMMERFELD}      # library boundary-condition codes -> the oracle's


def relres(n, bc, k, F, U):
    prob = Problem(n, OBC.get(bc, bc), k * k)
    A = prob.assemble_fast()
    out = []
    for f, u in zip(F.cpu().numpy(), U.cpu().numpy()):
        fv, uv = prob.grid_to_vec(f), prob.grid_to_vec(u)
        out.append(np.linalg.norm(fv - A @ uv) / np.linalg.norm(fv))
    return np.array(out)


def reldiff(a, b):
    return (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()


def same_results(U0, R0, U1, R1):
    assert [r.iterations for r in R1] == [r.iterations for r in R0]
    assert [r.converged for r in R1] == [r.converged for r in R0]
    for a, b in zip(R0, R1):
        assert abs(a.relres_est - b.relres_est) <= 1e-12 * max(a.relres_est, 1e-300)
        assert abs(a.relres_true - b.relres_true) <= 1e-12 * max(a.relres_true, 1e-300)
    assert reldiff(U1, U0) <= 1e-12


# (precision, orth_fp64, basis_df): FP64 CGS2; mixed with the delayed CGS2 on the
# complex128 basis; on the double-float basis; mixed with the all-FP64 CGS2
PATHS = [(0, False, False), (1, False, False), (1, False, True), (1, True, False)]


@pytest.mark.parametrize("prec,orth,df", PATHS)
def test_graph_solve_equals_stream_solve(hzs, prec, orth, df):
    n, k = 129, 25.0
    g = hzs.Grid(n, hzs.SOMMERFELD, k=k, nsub=4, overlap=2)
    P = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 16, prec)
    F = sources(n, 5, seed=21)
    U0, R0 = P.solve(F, tol=1e-8, maxit=300, orth_fp64=orth, basis_df=df)
    for _ in range(2):                                            # second call reuses the graphs
        U1, R1 = P.solve(F, tol=1e-8, maxit=300, orth_fp64=orth, basis_df=df, graph=True)
        torch.cuda.synchronize()
        same_results(U0, R0, U1, R1)
    assert all(r.converged for r in R1)
    assert np.all(relres(n, SOMMERFELD, k, F, U1) <= 1.01e-8)


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_solve_stopped_by_maxit_inside_a_chunk(hzs, prec):
    n, k = 65, 20.0
    g = hzs.Grid(n, hzs.DIRICHLET, k=k, nsub=4, overlap=2)
    P = hzs.Preconditioner(g, hzs.AS1, hzs.COARSE_NONE, 2, prec)
    f = torch.from_numpy(point_source(n)).cuda()
    U0, R0 = P.solve(f, tol=1e-14, maxit=13)
    U1, R1 = P.solve(f, tol=1e-14, maxit=13, graph=True)
    assert R0[0].iterations == 13 and not R0[0].converged
    same_results(U0, R0, U1, R1)


def test_graph_adjoint_solve_equals_stream(hzs):
    n, k = 129, 25.0
    g = hzs.Grid(n, hzs.SOMMERFELD, k=k, nsub=4, overlap=2)
    P = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 16, hzs.MIXED)
    rhs = torch.from_numpy(random_complex_grid(n, seed=5)).cuda()
    L0, R0 = P.adjoint_solve(rhs, tol=1e-8, maxit=300)
    L1, R1 = P.adjoint_solve(rhs, tol=1e-8, maxit=300, graph=True)
    same_results(L0, R0, L1, R1)


def test_graph_batched_problems_equal_stream(hzs):
    probs, rhs = [], []
    for (n, k, ns, p, cnt, seed) in [(65, 10.0, 2, 8, 3, 1), (129, 25.0, 4, 16, 4, 2)]:
        g = hzs.Grid(n, hzs.SOMMERFELD, k=k, nsub=ns, overlap=2, stream=torch.cuda.Stream())
        probs.append(hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, p, hzs.MIXED))
        rhs.append(sources(n, cnt, seed))
    torch.cuda.synchronize()
    outs0, res0 = hzs.solve_batched(probs, rhs, tol=1e-7, maxit=300)
    outs1, res1 = hzs.solve_batched(probs, rhs, tol=1e-7, maxit=300, graph=True)
    torch.cuda.synchronize()
    for U0, R0, U1, R1 in zip(outs0, res0, outs1, res1):
        same_results(U0, R0, U1, R1)


SHAPES_T = (1, 2)
SHAPES_NST = (1, 2, 4)
SHAPES_TPR = (4, 8)


@pytest.mark.parametrize("prec,bc,kind", [(0, 0, 3), (1, 0, 3), (1, 1, 2), (0, 1, 1)])
def test_autotuned_apply_equals_default(hzs, prec, bc, kind):
    n, k, nsub, p = 257, 20.0, 4, 32
    g = hzs.Grid(n, bc, k=k, nsub=nsub, overlap=2)
    P0 = hzs.Preconditioner(g, kind, hzs.COARSE_B2, p, prec)
    P1 = hzs.Preconditioner(g, kind, hzs.COARSE_B2, p, prec, autotune=2)
    i0, i1 = P0.info(), P1.info()
    assert i0["autotuned"] == 0 and i1["autotuned"] == 1
    for i in (i0, i1):
        assert i["tile_group"] in SHAPES_T and i["tile_stages"] in SHAPES_NST
        assert i["tile_threads_per_row"] in SHAPES_TPR
    assert 0.0 < i1["apply_us_tuned"] <= i1["apply_us_default"]
    assert i0["nfactors"] == i1["nfactors"] and i0["coarse_unknowns"] == i1["coarse_unknowns"]
    V = torch.from_numpy(random_complex_grid(n, seed=7, nrhs=3)).cuda()
    z0, z1 = P0.apply(V), P1.apply(V)
    torch.cuda.synchronize()
    assert reldiff(z1, z0) <= (1e-11 if prec == 0 else 1e-4)
    # solves with the default and the tuned shape
    f = torch.from_numpy(point_source(n)).cuda()
    _, r0 = P0.solve(f, tol=1e-7, maxit=1000)
    u, r = P1.solve(f, tol=1e-7, maxit=1000)
    assert r[0].converged == r0[0].converged
    assert abs(r[0].iterations - r0[0].iterations) <= (1 if prec == 0 else 3)
    if r[0].converged:
        assert relres(n, bc, k, f[None], u[None])[0] <= 1.01e-7
    # autotune = 1 reuses the choice made for the same problem
    P2 = hzs.Preconditioner(g, kind, hzs.COARSE_B2, p, prec, autotune=1)
    i2 = P2.info()
    assert i2["autotuned"] == 1
    assert (i2["tile_group"], i2["tile_stages"], i2["tile_threads_per_row"]) == \
        (i1["tile_group"], i1["tile_stages"], i1["tile_threads_per_row"])
    for P in (P0, P1, P2):
        P.close()
    g.close()


def test_autotune_rejects_bad_value(hzs):
    g = hzs.Grid(65, hzs.DIRICHLET, k=10.0, nsub=4, overlap=2)
    with pytest.raises(hzs.HzsError) as ei:
        hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 8, 0, autotune=3)
    assert ei.value.status == hzs.ERR_INVALID_ARG
