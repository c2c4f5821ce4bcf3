"""The library's Lorenz-Mie tables, full and chopped (host code of the CUDA library,
computed independently of the oracle's), equal the oracle's: the tracking kernels evaluate
and sample the same phase functions the oracle renders with.  No GPU needed."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1709_05418_gb300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    from paper_1709_05418_gb300 import build
    import torch  # noqa: F401  (shares the CUDA runtime with the library)
    L = ctypes.CDLL(build.build())
    dp = ctypes.POINTER(ctypes.c_double)
    L.rpnn_lorenz_mie_table.argtypes = [ctypes.c_int32, dp, dp, dp, ctypes.c_int32, dp]
    return L


def library_table(L, chopped, n=1800):
    p, cdf, ce, f = np.zeros(n), np.zeros(n + 1), np.zeros(n + 1), np.zeros(1)
    dp = ctypes.POINTER(ctypes.c_double)
    st = L.rpnn_lorenz_mie_table(chopped, p.ctypes.data_as(dp), cdf.ctypes.data_as(dp), ce.ctypes.data_as(dp),
                                 n, f.ctypes.data_as(dp))
    assert st == 0
    return p, cdf, ce, float(f[0])


def test_library_table_equals_oracle(lib):
    from paper_1709_05418_gb300 import api
    assert api.LM_BINS == oracle.LM_BINS and api.LM_CHOP_BINS == oracle.LM_CHOP_BINS
    p, cdf, ce, _ = library_table(lib, 0)
    rp, rcdf, rce = oracle.lm_table()
    assert np.allclose(p, rp, rtol=1e-9, atol=0), float(np.max(np.abs(p / rp - 1)))
    assert np.allclose(cdf, rcdf, rtol=0, atol=1e-12)
    assert np.allclose(ce, rce, rtol=0, atol=1e-15)
    # the kernels' FP32 copy keeps the forward peak and the tail to FP32 rounding
    assert np.allclose(p.astype(np.float32), rp, rtol=1e-7, atol=0)


def test_library_chopped_table_equals_oracle(lib):
    p, cdf, ce, f = library_table(lib, 1)
    v = oracle.Volume(W.blob_cloud(16, seed=1))
    v.set_phase(2)
    rp, rcdf = v.lm_chopped_table()
    rf = v.chop_params()[0]
    v.close()
    assert abs(f - rf) < 1e-11
    assert np.all((p == 0) == (rp == 0))
    assert np.allclose(p, rp, rtol=1e-9, atol=0)
    assert np.allclose(cdf, rcdf, rtol=0, atol=1e-12)
    assert np.allclose(ce, oracle.lm_table()[2], rtol=0, atol=1e-15)


def test_library_table_rejects_other_sizes(lib):
    assert lib.rpnn_lorenz_mie_table(0, None, None, None, 900, None) == -1
    assert lib.rpnn_lorenz_mie_table(1, None, None, None, 1800, None) == 0
