"""Full-size checks of the CUDA path at the sizes the benchmark runs (needs a GB300).

MP-1, k = 100, n = 1025 (16 x 16 subdomains, overlap 2, SHS2 / B_2 with H = 1/32,
tol 1e-6), in both precisions, and in the benchmark's configuration (mixed precision,
graph-issued Arnoldi steps, autotuned subdomain-solve shape):
  * the operator and one preconditioner apply equal the oracle's, element by
    element (oracle set-up at this size takes seconds);
  * the returned u has ||f - A u|| <= tol ||f|| with the oracle's matrix;
  * at 16 sampled nodes u is within the rigorous bound of the exact discrete
    solution, which the sine series gives node by node: A is real symmetric
    for MP-1, so ||u - u*||_2 <= ||f - A u||_2 / min |lambda_pq|.
MP-2, k = 50, n = 513 (8 x 8 subdomains, overlap 2, H = 1/16, tol 1e-7):
  * SHS2 / B_2 FP64: iteration count within 1 of the oracle's GMRES and the
    solution within 1e-5 of the oracle's; MIXED reaches tol with the
    mixed-precision step bar;
  * SHS2 / P_1 and one-level AS: preconditioner parity and residual.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import AS1, B2, DIRICHLET, P1, SHS2, SOMMERFELD, Problem, Schwarz, gmres  # noqa: E402
from paper_2408_03571_gb300.inputs import distinct_interior_nodes, point_source, random_complex_grid  # noqa: E402

pytestmark = pytest.mark.gpu


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
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def sine_series_at(n, k, nodes):
    """Exact discrete MP-1 solution for the centre source 1/h^2 at the given nodes."""
    N = n - 1
    h = 1.0 / N
    c = N // 2
    modes = np.arange(1, N)
    lam1 = (4.0 / h**2) * np.sin(modes * np.pi * h / 2) ** 2
    lam = lam1[:, None] + lam1[None, :] - k * k              # [q, p]
    sc = np.sqrt(2.0 / N) * np.sin(np.pi * modes * c / N)
    coef = np.outer(sc, sc) / (h * h * lam)                  # [q, p]
    out = []
    for (i, j) in nodes:
        si = np.sqrt(2.0 / N) * np.sin(np.pi * modes * i / N)
        sj = np.sqrt(2.0 / N) * np.sin(np.pi * modes * j / N)
        out.append(sj @ coef @ si)
    return np.array(out), np.min(np.abs(lam))


@pytest.fixture(scope="module")
def mp1_full():
    n, k = 1025, 100.0
    prob = Problem(n, DIRICHLET, k * k)
    A = prob.assemble_fast()
    M = Schwarz(prob, A, 16, 2, SHS2, B2, 32)
    return n, k, prob, A, M


# (precision, issue): FP64 and mixed stream-issued with the default subdomain-solve shape,
# and the benchmark's own configuration: mixed, graph-issued steps, autotuned shape
@pytest.mark.parametrize("prec,bench_cfg", [(0, False), (1, False), (1, True)],
                         ids=["fp64", "mixed", "mixed-graph-autotune"])
def test_mp1_headline_size(hzs, mp1_full, prec, bench_cfg):
    n, k, prob, A, M = mp1_full
    g = hzs.Grid(n, hzs.DIRICHLET, k=k, nsub=16, overlap=2)
    P = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 32, prec, autotune=1 if bench_cfg else 0)
    v = random_complex_grid(n, seed=77)
    vd = dev(v)
    y = P.apply_operator(vd).cpu().numpy()
    assert rel(prob.grid_to_vec(y), A @ prob.grid_to_vec(v)) < 1e-13
    z = P.apply(vd).cpu().numpy()
    zr = M.apply(prob.grid_to_vec(v))
    assert rel(prob.grid_to_vec(z), zr) < (1e-9 if prec == 0 else 1e-4)
    f = point_source(n)
    u, info = P.solve(dev(f), tol=1e-6, maxit=1000, graph=bench_cfg)
    assert info[0].converged
    uv = prob.grid_to_vec(u.cpu().numpy())
    fv = prob.grid_to_vec(f)
    r = np.linalg.norm(fv - A @ uv)
    assert r <= 1.01e-6 * np.linalg.norm(fv)
    nodes = distinct_interior_nodes(n, 16, seed=78) + [((n - 1) // 2, (n - 1) // 2)]
    exact, lam_min = sine_series_at(n, k, nodes)
    bound = r / lam_min
    got = np.array([u[j, i].item() for (i, j) in nodes])
    assert np.all(np.abs(got - exact) <= 1.01 * bound + 1e-12 * np.abs(exact).max())


@pytest.fixture(scope="module")
def mp2_half():
    n, k = 513, 50.0
    prob = Problem(n, SOMMERFELD, k * k)
    A = prob.assemble_fast()
    return n, k, prob, A


def test_mp2_shs2_b2_matches_oracle_solve(hzs, mp2_half):
    n, k, prob, A = mp2_half
    M = Schwarz(prob, A, 8, 2, SHS2, B2, 16)
    f = point_source(n)
    ref = gmres(lambda x: A @ x, M.apply, prob.grid_to_vec(f), 1e-7, 400)
    assert ref.converged
    g = hzs.Grid(n, hzs.SOMMERFELD, k=k, nsub=8, overlap=2)
    for prec in (0, 1):
        P = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 16, prec)
        u, info = P.solve(dev(f), tol=1e-7, maxit=400)
        assert info[0].converged
        if prec == 0:
            assert abs(info[0].iterations - ref.iterations) <= 1
        else:
            assert ref.iterations - 1 <= info[0].iterations <= 1.15 * ref.iterations + 2
        uv = prob.grid_to_vec(u.cpu().numpy())
        fv = prob.grid_to_vec(f)
        assert np.linalg.norm(fv - A @ uv) <= 1.01e-7 * np.linalg.norm(fv)
        assert rel(uv, ref.x) < 1e-5
        P.close()


@pytest.mark.parametrize("kind,coarse", [(SHS2, P1), (AS1, None)])
def test_mp2_other_preconditioners(hzs, mp2_half, kind, coarse):
    n, k, prob, A = mp2_half
    M = Schwarz(prob, A, 8, 2, kind, coarse, 16)
    g = hzs.Grid(n, hzs.SOMMERFELD, k=k, nsub=8, overlap=2)
    hk = {SHS2: hzs.SHS2, AS1: hzs.AS1}[kind]
    hc = {P1: hzs.COARSE_P1, None: hzs.COARSE_NONE}[coarse]
    for prec in (0, 1):
        P = hzs.Preconditioner(g, hk, hc, 16, prec)
        v = random_complex_grid(n, seed=5)
        z = P.apply(dev(v)).cpu().numpy()
        assert rel(prob.grid_to_vec(z), M.apply(prob.grid_to_vec(v))) < (1e-9 if prec == 0 else 1e-4)
        f = point_source(n)
        u, info = P.solve(dev(f), tol=1e-7, maxit=1000)
        fv = prob.grid_to_vec(f)
        uv = prob.grid_to_vec(u.cpu().numpy())
        res = np.linalg.norm(fv - A @ uv) / np.linalg.norm(fv)
        if info[0].converged:
            assert res <= 1.01e-7
        else:
            assert info[0].iterations == 1000 and abs(res - info[0].relres_true) <= 1e-6 * max(res, 1e-30) + 1e-12
        P.close()
