"""The C ABI library builds for sm_103a, loads, and exports every symbol that
include/fks.h declares; argument errors are reported before any device work
(no GPU needed)."""
import ctypes as C

import numpy as np
import pytest

from paper_1212_3660_gb300 import build, fks


@pytest.fixture(scope="module")
def lib():
    build.build()
    return fks.lib()


def test_exports_every_declared_symbol(lib):
    names = fks.declared_symbols()
    assert {"fks_create", "fks_solve", "fks_op_grid", "fks_op_apply", "fks_precond_apply"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_version_and_error_string(lib):
    assert "sm_103a" in fks.fks_version()
    assert isinstance(fks.fks_last_error(), str)


def test_argument_errors_without_gpu(lib):
    out = C.c_void_p()
    nc = (C.c_int64 * 3)(4, 4, 1)
    h = (C.c_double * 3)(1.0, 1.0, 1.0)
    cond = np.ones(16)
    st = lib.fks_op_grid(None, 2, nc, h, cond.ctypes.data, cond.ctypes.data, 0xF, C.byref(out))
    assert st == fks.FKS_ERR_ARG
    st = lib.fks_solve(None, None, 1, None, 1, None, 1, None, None, None, None, None, None, None, None, None)
    assert st == fks.FKS_ERR_ARG
    assert "NULL" in fks.fks_last_error()
    assert lib.fks_op_size(None) == 0
    rp = np.array([0, 1, 2], np.int64)
    cl = np.array([0, 1], np.int32)
    v = np.ones(2)
    st = lib.fks_op_csr(None, 2, rp.ctypes.data, cl.ctypes.data, v.ctypes.data, rp.ctypes.data, cl.ctypes.data,
                        v.ctypes.data, C.byref(out))
    assert st == fks.FKS_ERR_ARG and not out.value


def test_no_gpu_create_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(fks.FksError):
        fks.fks_create(0)


def test_server_argument_errors_without_gpu(lib):
    out = C.c_void_p()
    assert lib.fks_server_create(None, 1 << 30, 2, C.byref(out)) == fks.FKS_ERR_ARG
    assert lib.fks_server_submit(None, None, None) == fks.FKS_ERR_ARG
    assert lib.fks_server_cancel(None, 1) == fks.FKS_ERR_ARG
