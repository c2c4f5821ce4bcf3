"""FP16 density grids (the batched-serving and large-cloud inputs) against the oracle.

The library widens an FP16 grid to FP32 on load; the oracle is built from the same FP16
values widened to FP32 on the host, so statistics, tracking majorants and mip levels are
bit-exact, and renders (FP32 and BF16 networks, single and batched) match the FP64 oracle
at the tolerances of the FP32-grid tests."""
import numpy as np
import pytest

import oracle
from paper_1709_05418_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BF16_REL = 1e-2


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_05418_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def ctx(api):
    c = api.Context()
    c.set_weights(torch.from_numpy(W.he_init(seed=2)).cuda())
    yield c
    c.close()


def _fp16_cloud(shape, seed):
    """Seeded fBm cloud stored as FP16; returns (FP16 array, its exact FP32 widening)."""
    d16 = W.fbm_cloud(shape=shape, seed=seed, coverage=0.35).astype(np.float16)
    return d16, d16.astype(np.float32)


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("shape,seed", [((48, 48, 48), 201), ((40, 24, 56), 202)])
def test_fp16_stats_mips_and_majorants_bit_exact(ctx, shape, seed):
    d16, d32 = _fp16_cloud(shape, seed)
    v = ctx.load_volume(torch.from_numpy(d16).cuda())
    ctx.build_mips(v)
    gi = ctx.get_volume_info(v)
    o = oracle.Volume(d32)
    oi = o.stats()
    assert gi["mean"] == oi["mean"] and gi["majorant"] == oi["majorant"] and gi["nonzero"] == oi["nonzero"]
    assert np.float32(gi["inv_mean_f"]) == np.float32(oi["inv_mean_f"])
    assert gi["mip_of_level"] == oi["mip_of_level"]
    for lv in sorted(set(oi["mip_of_level"]) | {0}):
        g = ctx.copy_mip_level(v, lv).cpu().numpy()
        r = o.mip_level(lv, f32=True)
        assert np.array_equal(g.view(np.uint32), r.view(np.uint32)), f"level {lv}"
    assert np.array_equal(ctx.copy_brick_majorants(v).cpu().numpy(), o.brick_majorants())
    o.close()


@pytest.fixture(scope="module")
def fp16_scene(ctx):
    d16, d32 = _fp16_cloud((64, 64, 64), 203)
    v = ctx.load_volume(torch.from_numpy(d16).cuda())
    ctx.build_mips(v)
    cam = W.camera(d32.shape, 48, 48, spp=1, seed=5, light_seed=6)
    return v, oracle.Volume(d32), cam


def test_fp16_grid_render_f32_matches_oracle(ctx, api, fp16_scene):
    v, orc, cam = fp16_scene
    params = W.he_init(seed=2).astype(np.float64)
    img, nq = ctx.render(v, cam, precision=api.F32, want_count=True)
    ctx.sync_status()
    got = img.cpu().numpy().ravel().astype(np.float64)
    ref = orc.render_pixels(cam, np.arange(got.size), params=params)
    tol = 1e-3 * np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max()) + 1e-7
    assert nq > 0.2 * got.size
    assert (np.abs(got - ref) <= tol).mean() >= 0.98


def test_fp16_grid_render_bf16_matches_oracle(ctx, api, fp16_scene):
    v, orc, cam = fp16_scene
    params = W.he_init(seed=2).astype(np.float64)
    got = ctx.render(v, cam, precision=api.BF16).cpu().numpy().ravel().astype(np.float64)
    ctx.sync_status()
    ref = orc.render_pixels(cam, np.arange(got.size), params=params)
    assert _rel_l2(got, ref) <= BF16_REL
    scale = np.maximum(np.abs(ref), np.median(np.abs(ref[ref > 0])))
    assert (np.abs(got - ref) <= 3e-2 * scale).mean() >= 0.98


def test_fp16_grids_batched_items_match_oracle(ctx, api):
    """Three FP16 clouds of uneven sizes and query counts in one batched call: each item's
    image against the FP64 oracle's render of that item."""
    params = W.he_init(seed=2).astype(np.float64)
    jobs, orcs = [], []
    for i, (shape, w, h, spp) in enumerate([((32, 32, 32), 20, 16, 1), ((56, 40, 48), 40, 36, 2),
                                            ((24, 48, 40), 28, 30, 1)]):
        d16, d32 = _fp16_cloud(shape, 210 + i)
        v = ctx.load_volume(torch.from_numpy(d16).cuda())
        ctx.build_mips(v)
        jobs.append((v, W.camera(d32.shape, w, h, spp=spp, seed=220 + i, light_seed=230 + i)))
        orcs.append(oracle.Volume(d32))
    imgs, counts = ctx.render_batch(jobs, want_counts=True)
    ctx.sync_status()
    assert all(n > 0 for n in counts)
    for img, (v, cam), orc in zip(imgs, jobs, orcs):
        got = img.cpu().numpy().ravel().astype(np.float64)
        ref = orc.render_pixels(cam, np.arange(got.size), params=params)
        assert _rel_l2(got, ref) <= BF16_REL
        scale = np.maximum(np.abs(ref), np.median(np.abs(ref[ref > 0])))
        assert (np.abs(got - ref) <= 3e-2 * scale).mean() >= 0.97
        orc.close()
