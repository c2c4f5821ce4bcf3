"""Batched serving: several clouds of different sizes, image sizes, sample counts, seeds
and lights rendered by one rpnn_render_batch call (one compacted descriptor launch, one
network launch, captured as a CUDA graph) give exactly the images and query counts of
separate rpnn_render calls; the captured graph is replayed while the item list is
unchanged and rebuilt when an item, a volume or the weights change."""
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
    ctx.set_weights(torch.from_numpy(W.he_init(seed=2)).cuda())
    vols, jobs = [], []
    shapes = [(24, 24, 24), (40, 32, 48), (32, 32, 32), (48, 40, 36)]
    for i, shp in enumerate(shapes):
        dens = (W.blob_cloud(shp[0], nblobs=6, seed=50 + i) if i % 2 == 0
                else W.fbm_cloud(shape=shp, seed=60 + i))
        v = ctx.load_volume(torch.from_numpy(np.ascontiguousarray(dens)).cuda())
        ctx.build_mips(v)
        vols.append(v)
        cam = W.camera(dens.shape, 24 + 8 * i, 20 + 6 * i, spp=1 + (i % 3), seed=70 + i, light_seed=80 + i)
        jobs.append((v, cam))
    yield api, ctx, jobs
    ctx.close()


def _separate(api, ctx, jobs):
    imgs, counts = [], []
    for v, cam in jobs:
        img, nq = ctx.render(v, cam, precision=api.BF16, want_count=True)
        imgs.append(img.clone())
        counts.append(nq)
    return imgs, counts


def test_batch_equals_separate_renders(env):
    api, ctx, jobs = env
    ref, ref_n = _separate(api, ctx, jobs)
    assert all(n > 0 for n in ref_n)
    out, n = ctx.render_batch(jobs, want_counts=True)
    ctx.sync_status()
    assert n == ref_n
    for a, b in zip(out, ref):
        assert torch.equal(a, b)
    # replay of the captured graph into the same images
    for img in out:
        img.fill_(-1.0)
    out2 = ctx.render_batch(jobs, images=out)
    ctx.sync_status()
    for a, b in zip(out2, ref):
        assert torch.equal(a, b)


def test_batch_follows_changed_items_and_weights(env):
    api, ctx, jobs = env
    jobs2 = list(jobs)
    v, cam = jobs2[1]
    jobs2[1] = (v, dict(cam, seed=cam["seed"] + 1))
    out = ctx.render_batch(jobs2)
    ref, _ = _separate(api, ctx, jobs2)
    for a, b in zip(out, ref):
        assert torch.equal(a, b)
    ctx.set_weights(torch.from_numpy(W.he_init(seed=9)).cuda())
    out = ctx.render_batch(jobs2, images=out)
    ref, _ = _separate(api, ctx, jobs2)
    ctx.sync_status()
    for a, b in zip(out, ref):
        assert torch.equal(a, b)
    ctx.set_weights(torch.from_numpy(W.he_init(seed=2)).cuda())


def test_batch_rejects_bad_lists(env):
    api, ctx, jobs = env
    with pytest.raises(api.RPNNError):
        ctx.render_batch([])
    with pytest.raises(api.RPNNError):
        ctx.render_batch([jobs[0]] * 33)
    with pytest.raises(api.RPNNError):
        ctx.render_batch([(999, jobs[0][1])])


@pytest.mark.parametrize("prec_name", ["BF16", "F32"])
def test_chunked_render_equals_single_chunk(env, prec_name):
    """A render whose descriptor/network stages run in chunks (here 1,000 queries) gives
    the image of the unchunked render bit for bit."""
    api, ctx, jobs = env
    prec = getattr(api, prec_name)
    v, cam = jobs[3]
    cam = dict(cam, width=64, height=56, spp=2)
    ref, nq = ctx.render(v, cam, precision=prec, want_count=True)
    ref = ref.clone()
    assert nq > 2500
    ctx.set_render_chunk(1000)
    try:
        out = ctx.render(v, cam, precision=prec)
        ctx.sync_status()
        assert torch.equal(out, ref)
    finally:
        ctx.set_render_chunk(0)
    with pytest.raises(api.RPNNError):
        ctx.set_render_chunk(5)
