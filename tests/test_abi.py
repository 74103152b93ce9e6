"""The C ABI library builds, loads without a GPU, and exports every call include/hzs.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hzs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hzs_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_03571_gb300 import build, hzs
    build.build()
    return hzs.load()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "hzs_solve" in names and "hzs_precond_setup" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_2408_03571_gb300 import hzs
    assert sorted(hzs.EXPORTS) == _declared()


def test_host_only_calls(lib):
    assert lib.hzs_version().startswith(b"hzs")
    assert lib.hzs_status_string(0) == b"ok"
    assert lib.hzs_status_string(-4) == b"singular subdomain matrix"
    assert lib.hzs_last_error(None) is not None


def test_invalid_grid_rejected_without_gpu(lib):
    from paper_2408_03571_gb300 import hzs
    h = ctypes.c_void_p()
    for n, nsub, ov in [(64, 4, 1), (65, 5, 1), (65, 4, 9), (65, 4, -1), (3, 1, 0)]:
        d = hzs.GridDesc(n, hzs.DIRICHLET, 10.0, None, nsub, ov)
        assert lib.hzs_grid_create(ctypes.byref(d), None, ctypes.byref(h)) == hzs.ERR_INVALID_ARG
        assert h.value is None
        assert len(lib.hzs_last_error(None)) > 0


def test_null_handles_rejected_without_gpu(lib):
    """Every entry point that takes a handle rejects NULL with HZS_ERR_INVALID_ARG before any CUDA call."""
    from paper_2408_03571_gb300 import hzs
    info = hzs.PrecondInfo()
    assert lib.hzs_precond_get_info(None, ctypes.byref(info)) == hzs.ERR_INVALID_ARG
    sd = hzs.SolveDesc(1e-6, 10, 0)
    si = (hzs.SolveInfo * 1)()
    assert lib.hzs_solve(None, ctypes.byref(sd), None, None, 1, si) == hzs.ERR_INVALID_ARG
    assert lib.hzs_adjoint_solve(None, ctypes.byref(sd), None, None, 1, si) == hzs.ERR_INVALID_ARG
    assert lib.hzs_apply_operator(None, None, None, 1) == hzs.ERR_INVALID_ARG
    assert lib.hzs_apply_precond(None, None, None, 1) == hzs.ERR_INVALID_ARG
    assert lib.hzs_apply_precond_noalloc(None, None, None, 1) == hzs.ERR_INVALID_ARG
    assert lib.hzs_kappa_gradient(None, None, None, None) == hzs.ERR_INVALID_ARG
    out = ctypes.c_void_p()
    d = hzs.PrecondDesc(hzs.SHS2, hzs.COARSE_B2, 4, hzs.FP64, 1, 0, 0)
    assert lib.hzs_precond_setup(None, ctypes.byref(d), ctypes.byref(out)) == hzs.ERR_INVALID_ARG
    assert out.value is None
    lib.hzs_precond_destroy(None)
    lib.hzs_grid_destroy(None)
