"""Failure detection without a GPU fault: a NaN parameter is rejected by rpnn_set_weights
(the previous weights stay), a forced tiny iteration cap truncates tracking and raises
RPNN_ERR_ITER_LIMIT at the next status read, and the context stays usable after both."""
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
    params = torch.from_numpy(W.he_init(seed=2)).cuda()
    ctx.set_weights(params)
    cam = W.camera(dens.shape, 24, 24, spp=1, seed=3, light_seed=4)
    yield api, ctx, vol, params, cam
    ctx.close()


def test_nan_weights_are_rejected_and_previous_weights_kept(env):
    api, ctx, vol, params, cam = env
    before = ctx.render(vol, cam, precision=api.F32).clone()
    bad = params.clone()
    bad[12345] = float("nan")
    with pytest.raises(api.RPNNError) as e:
        ctx.set_weights(bad)
    assert e.value.code == -6
    bad[12345] = float("inf")
    with pytest.raises(api.RPNNError):
        ctx.set_weights(bad)
    after = ctx.render(vol, cam, precision=api.F32)
    ctx.sync_status()
    assert torch.equal(before, after)


def test_forced_iteration_cap_raises_iter_limit_and_context_recovers(env):
    api, ctx, vol, params, cam = env
    ref = ctx.render(vol, cam, precision=api.F32, mode=api.MODE_SINGLE)
    ctx.sync_status()
    ctx.set_iteration_cap(vol, 2)
    ctx.render(vol, cam, precision=api.F32, mode=api.MODE_SINGLE)
    with pytest.raises(api.RPNNError) as e:
        ctx.sync_status()
    assert e.value.code == -5
    ctx.set_iteration_cap(vol, 0)
    again = ctx.render(vol, cam, precision=api.F32, mode=api.MODE_SINGLE)
    ctx.sync_status()
    assert torch.equal(ref, again)
