"""hzs_apply_precond_noalloc: the allocation-free SAS2 apply, through the C ABI.

It serves callers that may not allocate device memory when they apply the
preconditioner (hosts that forbid allocation after start-up, applications that
keep all device memory in their own pool).  It must give the same z = M^{-1} v
as hzs_apply_precond on two calls in a row (the work array it shares between
calls must not leak state from one call into the next), take no device memory
(the device's free memory is the same before and after a call), and reject what
does not fit its fixed work space.  This file is collected last.
"""
import ctypes as ct

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-13   # the relative bar of the operator parity tests; the kernels are the same


@pytest.fixture(scope="module")
def hzs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03571_gb300 import build
    build.build()
    from paper_2408_03571_gb300 import hzs as mod
    return mod


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return torch.from_numpy(a).cuda()


def _noalloc(hzs, P, v):
    z = torch.full_like(v, complex(np.nan, np.nan))
    st = hzs.load().hzs_apply_precond_noalloc(P.handle, ct.c_void_p(v.data_ptr()), ct.c_void_p(z.data_ptr()), 1)
    return st, z


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
def test_matches_apply_precond_twice(hzs, prec, bc):
    n, nsub, ov, p = 129, 4, 2, 16
    g = hzs.Grid(n, bc, k=25.0, nsub=nsub, overlap=ov)
    P = hzs.Preconditioner(g, hzs.SAS2, hzs.COARSE_B2, p, prec)
    _noalloc(hzs, P, _rand(n, 0))             # first call on the device: looks up the array's address
    torch.cuda.synchronize()
    for seed in (1, 2):                       # two calls in a row, different inputs
        v = _rand(n, seed)
        ref = P.apply(v)
        z = torch.full_like(v, complex(np.nan, np.nan))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = hzs.load().hzs_apply_precond_noalloc(P.handle, ct.c_void_p(v.data_ptr()), ct.c_void_p(z.data_ptr()), 1)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert st == hzs.OK
        err = (torch.linalg.vector_norm(z - ref) / torch.linalg.vector_norm(ref)).item()
        assert err < TOL
        if prec == 1:
            # the complex64 subdomain solve rounds each value once, where it stores it
            assert torch.equal(z, ref)


def test_rejects_what_does_not_fit(hzs):
    g = hzs.Grid(65, 0, k=10.0, nsub=4, overlap=2)
    P = hzs.Preconditioner(g, hzs.SHS2, hzs.COARSE_B2, 8, 0)
    st, _ = _noalloc(hzs, P, _rand(65, 3))
    assert st == hzs.ERR_INVALID_ARG
    assert b"SAS2" in hzs.load().hzs_last_error(g.handle)
    # work space n * nc1 * 16 B + 2 Nc * 16 B > 1 MiB
    g2 = hzs.Grid(1025, 0, k=10.0, nsub=16, overlap=2)
    P2 = hzs.Preconditioner(g2, hzs.SAS2, hzs.COARSE_B2, 16, 0)
    st, _ = _noalloc(hzs, P2, _rand(1025, 4))
    assert st == hzs.ERR_INVALID_ARG
    assert b"work space" in hzs.load().hzs_last_error(g2.handle)
