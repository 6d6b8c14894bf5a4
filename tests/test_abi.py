"""C-ABI checks that need no GPU: the library builds/loads, exports every declared symbol, and
rejects invalid arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2509_21064_gb300.build import build as build_lib
from paper_2509_21064_gb300 import sbo as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build_lib()
    return S.lib()


def declared_symbols():
    with open(os.path.join(ROOT, "include", "sbo.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sbo_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_what_the_binding_exports():
    assert declared_symbols() == sorted(S.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    for name in declared_symbols():
        assert hasattr(L, name), name
        assert ctypes.cast(getattr(L, name), ctypes.c_void_p).value


def test_version_and_empty_error(L):
    assert "sm_103a" in S.sbo_version()
    assert L.sbo_last_error() is not None


def test_invalid_arguments_are_rejected_without_a_device(L):
    out = ctypes.c_void_p()
    Q = np.zeros((4, 4), np.int32)
    qp = Q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    assert L.sbo_create_dense(0, qp, None, S.SBO_BF16, None, ctypes.byref(out)) == S.SBO_EINVAL
    assert L.sbo_create_dense(4, None, None, S.SBO_BF16, None, ctypes.byref(out)) == S.SBO_EINVAL
    assert L.sbo_create_dense(4, qp, None, S.SBO_FP8_E4M3, None, ctypes.byref(out)) == S.SBO_EINVAL
    assert b"FP8" in L.sbo_last_error()
    assert L.sbo_create_dense(4, qp, None, S.SBO_BF16, None, None) == S.SBO_EINVAL
    # malformed CSR: rowptr not monotone, column out of range
    rp = np.array([0, 2, 1, 3], np.int64)
    col = np.array([1, 2, 0], np.int32)
    val = np.array([1, 1, 1], np.int32)
    args = (rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            val.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    assert L.sbo_create_csr(3, 3, *args, None, S.SBO_FP32, None, ctypes.byref(out)) == S.SBO_EINVAL
    rp2 = np.array([0, 1, 2, 3], np.int64)
    col2 = np.array([1, 5, 0], np.int32)
    args2 = (rp2.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), col2.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
             val.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    assert L.sbo_create_csr(3, 3, *args2, None, S.SBO_FP32, None, ctypes.byref(out)) == S.SBO_EINVAL
    # weights not exact in E4M3 (|A_ij| = 2*17 > 16)
    col3 = np.array([1, 2, 0], np.int32)
    val3 = np.array([17, 1, 1], np.int32)
    args3 = (rp2.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), col3.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
             val3.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    assert L.sbo_create_csr(3, 3, *args3, None, S.SBO_FP8_E4M3, None, ctypes.byref(out)) == S.SBO_ERANGE
    # NULL handles
    prm = S.params(4, 10, 0.1, 0.1, 1.0)
    assert L.sbo_gda_start(None, ctypes.byref(prm), None) == S.SBO_EINVAL
    assert L.sbo_gda_run(None, 3) == S.SBO_EINVAL
    assert L.sbo_sync(None) == S.SBO_EINVAL
    assert L.sbo_best(None, None, None, None, None) == S.SBO_EINVAL
    assert L.sbo_set_option(None, 1, 0) == S.SBO_EINVAL
    assert L.sbo_launch_count(None) == 0
    L.sbo_destroy(None)


def test_valid_arguments_without_a_device_report_ecuda(L):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a device is present")
    except ImportError:
        pass
    out = ctypes.c_void_p()
    Q = np.zeros((4, 4), np.int32)
    st = L.sbo_create_dense(4, Q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), None, S.SBO_FP32, None,
                            ctypes.byref(out))
    assert st == S.SBO_ECUDA
    assert out.value is None


def test_params_default_grad_tol_is_two_delta():
    p = S.params(8, 100, 0.1, 0.2, 3.0, delta=0.05)
    assert p.grad_tol == pytest.approx(0.1)
    assert p.restarts == 8 and p.iters == 100 and p.eval_every == 10
