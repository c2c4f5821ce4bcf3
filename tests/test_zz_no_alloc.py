"""rpnn_mlp_forward_f32_static: the FP32 network forward for callers that cannot call
cudaMalloc while they run it (device memory owned by their own allocator or reserved up
front under a fixed budget, real-time loops that allow no allocation after start-up).  Its
scratch is a static device array and it runs the context path's own forward routine with
the default GEMM tile, so it must give bit for bit what the allocating entry point gives
(tile shapes change no result bit; forward GEMMs are never split along K), whether or not
the context tunes its tiles.  This file is collected last so a failure here comes after
every other test has run."""
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


def _static(L, params, zd, out, stream):
    return L.rpnn_mlp_forward_f32_static(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(zd.data_ptr()),
                                         zd.shape[0], ctypes.c_void_p(out.data_ptr()), stream)


@pytest.mark.parametrize("autotune", [False, True])
def test_static_forward_equals_allocating_forward_twice(lib, autotune):
    api, L = lib
    rng = np.random.default_rng(31)
    params = torch.from_numpy(W.he_init(seed=32, bias=0.02)).cuda()
    ctx = api.Context()
    ctx.set_weights(params)
    ctx.set_autotune(autotune)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for q in (4096, 777):                       # two calls in a row, the second smaller
        z = np.zeros((q, 10, 240), np.float32)
        z[:, :, :226] = rng.uniform(0, 2, size=(q, 10, 226))
        zd = torch.from_numpy(z).cuda()
        ref = ctx.mlp_forward(zd, precision=api.F32)
        out = torch.full((q,), float("nan"), dtype=torch.float32, device="cuda")
        rc = _static(L, params, zd, out, stream)
        assert rc == 0, L.rpnn_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert (ref > 0).float().mean() > 0.2
        assert torch.equal(out, ref), float((out - ref).abs().max())
    ctx.close()


def test_static_forward_takes_no_device_memory(lib):
    """After its first call on the device (which looks up the array's address), a call
    leaves the device's free memory where it was: it allocates nothing."""
    api, L = lib
    params = torch.from_numpy(W.he_init(seed=33)).cuda()
    z = torch.rand((1500, 10, 240), dtype=torch.float32, device="cuda")
    out = torch.empty(1500, dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert _static(L, params, z, out, stream) == 0, L.rpnn_last_error()
    torch.cuda.synchronize()
    first = out.clone()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _static(L, params, z, out, stream) == 0, L.rpnn_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 < (2 << 20), (free0, free1)     # below one allocation page
    assert torch.equal(out, first)


def test_static_forward_rejects_oversize(lib):
    api, L = lib
    rc = L.rpnn_mlp_forward_f32_static(ctypes.c_void_p(1), ctypes.c_void_p(1), 4097, ctypes.c_void_p(1), None)
    assert rc == -1
    assert b"at most 4096 rows" in L.rpnn_last_error()
