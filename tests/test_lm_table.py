"""The library's Lorenz-Mie table (host code of the CUDA library, computed independently of
the oracle's) equals the oracle's table: the tracking kernels evaluate and sample the same
phase function the oracle renders with.  No GPU needed."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1709_05418_gb300 import build
    import torch  # noqa: F401  (shares the CUDA runtime with the library)
    L = ctypes.CDLL(build.build())
    dp = ctypes.POINTER(ctypes.c_double)
    L.rpnn_lorenz_mie_table.argtypes = [dp, dp, dp, ctypes.c_int32]
    return L


def library_table(L, n=1800):
    p, cdf, ce = np.zeros(n), np.zeros(n + 1), np.zeros(n + 1)
    dp = ctypes.POINTER(ctypes.c_double)
    st = L.rpnn_lorenz_mie_table(p.ctypes.data_as(dp), cdf.ctypes.data_as(dp), ce.ctypes.data_as(dp), n)
    assert st == 0
    return p, cdf, ce


def test_library_table_equals_oracle(lib):
    import oracle
    from paper_1709_05418_gb300 import api
    assert api.LM_BINS == oracle.LM_BINS
    p, cdf, ce = library_table(lib)
    rp, rcdf, rce = oracle.lm_table()
    assert np.allclose(p, rp, rtol=1e-9, atol=0), float(np.max(np.abs(p / rp - 1)))
    assert np.allclose(cdf, rcdf, rtol=0, atol=1e-12)
    assert np.allclose(ce, rce, rtol=0, atol=1e-15)
    # the kernels' FP32 copy keeps the forward peak and the tail to FP32 rounding
    assert np.allclose(p.astype(np.float32), rp, rtol=1e-7, atol=0)


def test_library_table_rejects_other_sizes(lib):
    assert lib.rpnn_lorenz_mie_table(None, None, None, 900) == -1
    assert lib.rpnn_lorenz_mie_table(None, None, None, 1800) == 0
