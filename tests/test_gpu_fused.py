"""The render's descriptor gather fused into the BF16 tensor-core network (one kernel, no
descriptor rows in memory) against the unfused stages (k_descriptor, then k_rpnn_tc reading
the rows): the same FP32 descriptor arithmetic, BF16 rounding and MMA sequence, so the
images are equal bit for bit -- on a small cloud (a ragged last tile), on the 256^3 / 512x512
benchmark render (about 9 tiles per persistent block), over chunked renders (device-side
query counts) and under several lights; and the fused render against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1709_05418_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_05418_gb300 import api
    ctx = api.Context()
    params = W.he_init(seed=2)
    ctx.set_weights(torch.from_numpy(params).cuda())
    yield api, ctx, params
    ctx.close()


def _both(api, ctx, fn):
    ref = fn().clone()
    ctx.set_fused(True)
    try:
        got = fn().clone()
    finally:
        ctx.set_fused(False)
    ctx.sync_status()
    return got, ref


@pytest.mark.parametrize("shape,w,h,spp", [((64, 64, 64), 64, 64, 1), ((40, 24, 48), 37, 23, 3)])
def test_fused_render_equals_unfused(env, shape, w, h, spp):
    api, ctx, _ = env
    dens = W.blob_cloud(64, seed=1) if shape == (64, 64, 64) else W.fbm_cloud(shape=shape, seed=9, coverage=0.35)
    vol = ctx.load_volume(torch.from_numpy(dens).cuda())
    ctx.build_mips(vol)
    cam = W.camera(dens.shape, w, h, spp=spp, seed=3, light_seed=4)
    got, ref = _both(api, ctx, lambda: ctx.render(vol, cam, precision=api.BF16))
    assert (ref > 0).float().mean() > 0.2
    assert torch.equal(got, ref)


def test_fused_benchmark_render_equals_unfused(env):
    api, ctx, _ = env
    dens = W.fbm_cloud(256, seed=7)
    vol = ctx.load_volume(torch.from_numpy(dens).cuda())
    ctx.build_mips(vol)
    cam = W.camera(dens.shape, 512, 512, spp=1, seed=3, light_seed=4)
    nq = {}

    def render():
        img, nq["q"] = ctx.render(vol, cam, precision=api.BF16, want_count=True)
        return img
    got, ref = _both(api, ctx, render)
    assert nq["q"] > 152 * 128 * 8            # several tiles per persistent block
    assert torch.equal(got, ref)


def test_fused_chunked_and_env_renders_equal_unfused(env):
    api, ctx, _ = env
    dens = W.blob_cloud(64, seed=1)
    vol = ctx.load_volume(torch.from_numpy(dens).cuda())
    ctx.build_mips(vol)
    cam = W.camera(dens.shape, 48, 40, spp=2, seed=5, light_seed=6)
    ctx.set_render_chunk(1000)                # several chunks with device-side counts
    try:
        got, ref = _both(api, ctx, lambda: ctx.render(vol, cam, precision=api.BF16))
        assert torch.equal(got, ref)
    finally:
        ctx.set_render_chunk(0)
    rng = np.random.default_rng(12)
    dirs = rng.normal(size=(5, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    irr = rng.uniform(0.2, 1.0, size=5)
    got, ref = _both(api, ctx, lambda: ctx.render_env(vol, cam, dirs, irr, precision=api.BF16))
    assert torch.equal(got, ref)


def test_fused_render_matches_oracle(env):
    api, ctx, params = env
    dens = W.fbm_cloud(shape=(48, 56, 40), seed=21, coverage=0.35)
    vol = ctx.load_volume(torch.from_numpy(dens).cuda())
    ctx.build_mips(vol)
    cam = W.camera(dens.shape, 40, 40, spp=1, seed=7, light_seed=8)
    ctx.set_fused(True)
    try:
        got = ctx.render(vol, cam, precision=api.BF16).cpu().numpy().ravel().astype(np.float64)
        ctx.sync_status()
    finally:
        ctx.set_fused(False)
    ref = oracle.Volume(dens).render_pixels(cam, np.arange(got.size), params=params.astype(np.float64))
    assert float(np.linalg.norm(got - ref) / np.linalg.norm(ref)) <= 1e-2
    scale = np.maximum(np.abs(ref), np.median(np.abs(ref[ref > 0])))
    assert (np.abs(got - ref) <= 3e-2 * scale).mean() >= 0.98
