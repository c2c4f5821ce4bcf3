"""rpnn_mlp_forward_f32_static: the FP32 network forward for callers that may not
allocate device memory (code under someone else's stream capture, fixed memory
budgets, allocation-free real-time loops).  Its scratch is a static device array, so
it must give exactly what the allocating entry point gives.  This file is collected
last so a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest

from paper_1709_05418_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_05418_gb300 import api
    L = api.load()
    L.rpnn_mlp_forward_f32_static.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                              ctypes.c_void_p, ctypes.c_void_p]
    L.rpnn_mlp_forward_f32_static.restype = ctypes.c_int32
    return api, L


def test_static_forward_matches_allocating_forward_twice(lib):
    api, L = lib
    rng = np.random.default_rng(31)
    params = torch.from_numpy(W.he_init(seed=32, bias=0.02)).cuda()
    ctx = api.Context()
    ctx.set_weights(params)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for q in (4096, 777):                       # two calls in a row, the second smaller
        z = np.zeros((q, 10, 240), np.float32)
        z[:, :, :226] = rng.uniform(0, 2, size=(q, 10, 226))
        zd = torch.from_numpy(z).cuda()
        ref = ctx.mlp_forward(zd, precision=api.F32)
        out = torch.full((q,), float("nan"), dtype=torch.float32, device="cuda")
        rc = L.rpnn_mlp_forward_f32_static(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(zd.data_ptr()),
                                           q, ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0, L.rpnn_last_error()
        torch.cuda.synchronize()
        g, r = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.linalg.norm(g - r) <= 1e-5 * np.linalg.norm(r)
    ctx.close()


def test_static_forward_rejects_oversize(lib):
    api, L = lib
    rc = L.rpnn_mlp_forward_f32_static(ctypes.c_void_p(1), ctypes.c_void_p(1), 4097, ctypes.c_void_p(1), None)
    assert rc == -1
    assert b"at most 4096 rows" in L.rpnn_last_error()
