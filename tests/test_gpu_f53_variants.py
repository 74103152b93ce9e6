"""Every launch variant of the f53 passes (the FP64 Arnoldi of the mixed path, delayed
CGS2 on a basis stored as FP32 heads and 29-bit tails) computes the same FP64 Arnoldi
process, through the C ABI.

The variants differ only in which vectors are summed with FP64 multiply-adds and which
in FP32 three-word expansions (the vector masks), in how the dot pass assigns vectors to
warps (mixed tasks of 1 or 2 vectors, with or without a shared-memory copy ring, or
tasks specialised to one path) and in blocks per SM.  Each is selected by the HZS_F53_*
variables, read when the solve's work space is made, and must reproduce the run of the
four-pass FP64 CGS2 under the same complex64 preconditioner:

* at tol 1e-12: the same step count within one, the true residual at tol, the GMRES
  estimate equal to the true residual to 1e-2 of it (the Arnoldi relation holds to FP64
  rounding), and the solution within 1e-9 of the FP64 CGS2's;
* on a ragged size (n = 97: N = 9409 entries, not a multiple of the block chunks) and
  with masks that put every vector on one path (0x00, 0xFF).
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2408_03571_gb300.inputs import point_source  # noqa: E402

pytestmark = pytest.mark.gpu

KNOBS = ("HZS_F53_MASK", "HZS_F53_OCC", "HZS_F53_DOT_OCC", "HZS_F53_WS", "HZS_F53_GROUP", "HZS_F53_RING",
         "HZS_F53_UPD_E", "HZS_F53_G64", "HZS_F53_RING64", "HZS_F53_DOT_WAVES")

VARIANTS = [
    {},                                                                     # the defaults
    {"HZS_F53_WS": "0", "HZS_F53_RING": "0", "HZS_F53_GROUP": "2", "HZS_F53_DOT_OCC": "3"},
    {"HZS_F53_WS": "0", "HZS_F53_RING": "4", "HZS_F53_GROUP": "1", "HZS_F53_DOT_OCC": "4"},
    {"HZS_F53_WS": "0", "HZS_F53_RING": "3", "HZS_F53_GROUP": "2", "HZS_F53_DOT_OCC": "2"},
    {"HZS_F53_WS": "1", "HZS_F53_GROUP": "1", "HZS_F53_DOT_OCC": "3"},
    {"HZS_F53_MASK": "0x00,0x00"},                                          # every vector on the FP32 path
    {"HZS_F53_MASK": "0xFF,0xFF"},                                          # every vector on the FP64 path
    {"HZS_F53_MASK": "0x11,0x55", "HZS_F53_OCC": "2"},
    {"HZS_F53_MASK": "0x00,0xFF", "HZS_F53_WS": "0"},
    {"HZS_F53_UPD_E": "1", "HZS_F53_OCC": "3", "HZS_F53_MASK": "0x6D,0x77"},
    {"HZS_F53_G64": "8", "HZS_F53_GROUP": "2"},
    {"HZS_F53_UPD_E": "2", "HZS_F53_OCC": "3"},
    {"HZS_F53_RING64": "1"},
    {"HZS_F53_RING64": "1", "HZS_F53_MASK": "0xFF,0x6D"},
    {"HZS_F53_MASK": "0x6D,0xFF"},
    {"HZS_F53_MASK": "0x6D,0x00"},
    {"HZS_F53_DOT_WAVES": "2"},
]


@pytest.fixture(scope="module")
def hzs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03571_gb300 import build
    build.build()
    from paper_2408_03571_gb300 import hzs as mod
    return mod


@pytest.fixture
def knobs():
    saved = {k: os.environ.get(k) for k in KNOBS}
    yield
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


def _solve(hzs, n, bc, k, nsub, p, tol, env, **kw):
    for key in KNOBS:
        os.environ.pop(key, None)
    os.environ.update(env)
    g = hzs.Grid(n, bc, k=k, nsub=nsub, overlap=2)
    P = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, p, hzs.MIXED)
    f = torch.from_numpy(point_source(n)).cuda()
    u, info = P.solve(f, tol=tol, maxit=400, **kw)
    out = u.cpu().numpy(), info[0]
    P.close()
    g.close()
    return out


@pytest.mark.parametrize("env", VARIANTS, ids=lambda e: ",".join(f"{k[8:]}={v}" for k, v in e.items()) or "default")
@pytest.mark.parametrize("n,bc,k,nsub,p", [(129, 1, 25.0, 4, 16), (97, 0, 18.0, 4, 8)])
def test_variant_is_the_fp64_arnoldi(hzs, knobs, env, n, bc, k, nsub, p):
    tol = 1e-12
    u_ref, i_ref = _solve(hzs, n, bc, k, nsub, p, tol, {}, orth_fp64=True)
    u, info = _solve(hzs, n, bc, k, nsub, p, tol, env)
    assert info.orth_kind == hzs.ORTH_DCGS2_FP64          # the f53 basis (FP64 and FP32 pipes)
    assert info.converged and abs(info.iterations - i_ref.iterations) <= 1
    assert info.relres_true <= 1.01 * tol
    assert abs(info.relres_est - info.relres_true) <= 1e-2 * info.relres_true + 1e-15
    assert np.linalg.norm(u - u_ref) <= 1e-9 * np.linalg.norm(u_ref)
