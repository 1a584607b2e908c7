"""The tcgen05 building block (include/sv_selftest.h) against a host product.

The tensor core reads FP32 inputs of kind::tf32 with the low 13 mantissa bits
dropped; the reference does the same truncation and multiplies in FP64, so
only the FP32 accumulation order differs."""
import ctypes

import numpy as np
import pytest

import paper_2504_03967_gb300 as S
from paper_2504_03967_gb300 import build as B

pytestmark = pytest.mark.gpu


def tf32(x):
    return (x.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)


def test_tc_tf32_product():
    B.build()
    f = S.lib().sv_selftest_tc_tf32
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int] * 3 + [ctypes.c_void_p]
    f.restype = ctypes.c_int
    rng = np.random.default_rng(5)
    A = rng.standard_normal((128, 64)).astype(np.float32)
    Bm = rng.standard_normal((64, 64)).astype(np.float32)
    D = np.zeros((128, 64), np.float32)
    st = ctypes.c_int(-1)
    rc = f(A.ctypes.data, Bm.ctypes.data, D.ctypes.data, 128, 2048, 0, ctypes.byref(st))
    assert rc == 0, S.sv_last_error()
    assert st.value == 0
    ref = tf32(A).astype(np.float64) @ tf32(Bm).astype(np.float64).T
    assert np.abs(D - ref).max() < 1e-4
    # the untruncated product differs by far more: the check above is sharp
    assert np.abs(A.astype(np.float64) @ Bm.astype(np.float64).T - ref).max() > 1e-3


def test_tc_f16_product():
    """kind::f16 with A in tensor memory: FP16 inputs are exact, so the product
    equals the FP64 product of the same FP16 values up to FP32 accumulation;
    the swapped half-word order gives a different, wrong product."""
    B.build()
    f = S.lib().sv_selftest_tc_f16
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_void_p]
    f.restype = ctypes.c_int
    rng = np.random.default_rng(6)
    A = rng.standard_normal((128, 64)).astype(np.float16)
    Bm = rng.standard_normal((64, 64)).astype(np.float16)
    ref = A.astype(np.float64) @ Bm.astype(np.float64).T
    out = {}
    for swap in (0, 1):
        D = np.zeros((128, 64), np.float32)
        st = ctypes.c_int(-1)
        rc = f(A.view(np.uint16).ctypes.data, Bm.view(np.uint16).ctypes.data, D.ctypes.data, swap, ctypes.byref(st))
        assert rc == 0, S.sv_last_error()
        assert st.value == 0
        out[swap] = np.abs(D - ref).max()
    assert out[0] < 1e-4, out
    assert out[1] > 1e-2, out
