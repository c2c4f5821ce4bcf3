"""Training on the GPU (Sec. 5) and what the trained network gains (Sec. 4.4, Sec. 6):
records are path traced by the library, the network is fitted with the library's own
forward/backward kernels, and a render of a held-out cloud with the trained network is
closer to a converged path-traced reference than the method without the network
(single scattering only, L_i = 0)."""
import numpy as np
import pytest

from paper_1709_05418_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_05418_gb300 import api, train
    ctx = api.Context()
    yield api, train, ctx
    ctx.close()


def test_training_reduces_loss_and_beats_single_scattering(env):
    api, train, ctx = env
    clouds = train.blob_clouds(4, size=48, seed0=300)
    desc, label = train.records(ctx, clouds, 6000, seed=11, rel_ci=0.1, n_min=32, n_max=512)
    assert desc.shape == (24000, 10, 240) and torch.isfinite(label).all()
    assert (label > 0).float().mean() > 0.5
    tr, va = train.split(desc, label)
    params = torch.from_numpy(W.he_init(seed=5)).cuda()
    params.mul_(0.5)
    ctx.set_weights(params)
    v0 = train.val_loss(ctx, *va)
    hist = train.fit(ctx, tr, va, params, steps=400, batch=1024, lr=1e-3, eval_every=100)
    v1 = hist[-1][2]
    assert v1 < 0.25 * v0, (v0, hist)
    # held-out cloud, reference by plain path tracing
    held = W.blob_cloud(48, nblobs=8, seed=999)
    vol = ctx.load_volume(torch.from_numpy(held).cuda())
    ctx.build_mips(vol)
    cam = W.camera(held.shape, 40, 40, spp=8, seed=12, light_seed=13)
    ref_cam = dict(cam, spp=512)
    ref = ctx.render(vol, ref_cam, mode=api.MODE_PATH).double()
    ctx.set_weights(params)
    rp = ctx.render(vol, cam, precision=api.F32, mode=api.MODE_RPNN).double()
    ss = ctx.render(vol, cam, mode=api.MODE_SINGLE).double()
    ctx.sync_status()
    mask = ref > 0
    rmse_rpnn = float(torch.sqrt(((rp - ref)[mask] ** 2).mean()))
    rmse_ss = float(torch.sqrt(((ss - ref)[mask] ** 2).mean()))
    assert rmse_rpnn < 0.7 * rmse_ss, (rmse_rpnn, rmse_ss)
