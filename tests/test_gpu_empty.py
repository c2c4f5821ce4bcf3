"""Degenerate inputs: a camera that sees none of the cloud gives zero shading points, and
every stage (descriptor, tensor-core network with a device-side count of zero, scatter,
composite) runs through it: the image is exactly zero in every precision, under
environment lighting and inside a batch whose other item does hit the cloud."""
import numpy as np
import pytest

from paper_1709_05418_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_05418_gb300 import api
    ctx = api.Context()
    dens = W.blob_cloud(32, nblobs=6, seed=1)
    vol = ctx.load_volume(torch.from_numpy(dens).cuda())
    ctx.build_mips(vol)
    ctx.set_weights(torch.from_numpy(W.he_init(seed=2)).cuda())
    cam = W.camera(dens.shape, 40, 30, spp=2, seed=3, light_seed=4)
    away = dict(cam, cam_fwd=tuple(-np.asarray(cam["cam_fwd"])), cam_right=tuple(-np.asarray(cam["cam_right"])))
    yield api, ctx, vol, cam, away
    ctx.close()


def test_render_with_no_shading_point(env):
    api, ctx, vol, cam, away = env
    for prec in (api.F32, api.BF16):
        img, nq = ctx.render(vol, away, precision=prec, want_count=True)
        ctx.sync_status()
        assert nq == 0 and float(img.abs().max()) == 0.0
    # FP8 once calibrated on some shading points of the visible view
    hit, x, d, _ = ctx.trace_primary(vol, cam)
    idx = torch.nonzero(hit).squeeze(1)
    wl = torch.tensor(cam["light_dir"], dtype=torch.float32, device="cuda")
    ctx.calibrate_fp8(ctx.extract_descriptors(vol, x[idx].contiguous(), d[idx].contiguous(), wl))
    img8, nq8 = ctx.render(vol, away, precision=api.FP8, want_count=True)
    ctx.sync_status()
    assert nq8 == 0 and float(img8.abs().max()) == 0.0
    dirs = np.array([cam["light_dir"], (0.0, 1.0, 0.0)], np.float32)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    ie = ctx.render_env(vol, away, dirs, [1.0, 0.3], precision=api.BF16)
    ctx.sync_status()
    assert float(ie.abs().max()) == 0.0


def test_batch_with_an_empty_item(env):
    api, ctx, vol, cam, away = env
    images, counts = ctx.render_batch([(vol, away), (vol, cam)], want_counts=True)
    ctx.sync_status()
    assert counts[0] == 0 and counts[1] > 0
    assert float(images[0].abs().max()) == 0.0
    ref = ctx.render(vol, cam, precision=api.BF16)
    ctx.sync_status()
    assert torch.equal(images[1], ref)
