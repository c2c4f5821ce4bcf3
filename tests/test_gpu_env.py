"""Environment lighting (Sec. 4.4: a distant emitter approximated by directional samples):
rpnn_render_env against the sum of single-light renders of the library (same visible
points, same shadow streams, the same descriptor and network per light) and against the
FP64 oracle's environment render."""
import numpy as np
import pytest

from paper_1709_05418_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    from paper_1709_05418_gb300 import api
    ctx = api.Context()
    dens = W.blob_cloud(64, seed=1)
    vol = ctx.load_volume(torch.from_numpy(dens).cuda())
    ctx.build_mips(vol)
    params = W.he_init(seed=2)
    ctx.set_weights(torch.from_numpy(params).cuda())
    cam = W.camera((64, 64, 64), 48, 40, spp=2, seed=21, light_seed=22)
    # a "sun" and four "sky" directions of lower irradiance
    sky = [W.unit_sphere_dir(100 + i) for i in range(4)]
    dirs = np.array([cam["light_dir"]] + [s if s[1] > 0 else -s for s in sky], np.float32)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    irr = np.array([1.0, 0.15, 0.1, 0.2, 0.05], np.float32)
    yield api, ctx, vol, oracle.Volume(dens), params, cam, dirs, irr
    ctx.close()


def single_sum(api, ctx, vol, cam, dirs, irr, precision, mode):
    acc = None
    for w, e in zip(dirs, irr):
        cj = dict(cam, light_dir=tuple(float(v) for v in w), light_E=float(e))
        img = ctx.render(vol, cj, precision=precision, mode=mode).double()
        acc = img if acc is None else acc + img
    return acc


@pytest.mark.parametrize("precision,mode", [("F32", 0), ("BF16", 0), ("F32", 1)])
def test_env_render_is_sum_of_single_light_renders(env, precision, mode):
    api, ctx, vol, _, _, cam, dirs, irr = env
    prec = getattr(api, precision)
    got, nq = ctx.render_env(vol, cam, dirs, irr, precision=prec, mode=mode, want_count=True)
    ref = single_sum(api, ctx, vol, cam, dirs, irr, prec, mode)
    ctx.sync_status()
    got = got.double()
    assert float(ref.abs().max()) > 0
    # FP32 sums of the same terms in another order
    tol = 1e-5 * float(ref.abs().max()) + 1e-6 * ref.abs()
    assert bool(((got - ref).abs() <= tol).all()), float((got - ref).abs().max())
    if mode == 0:
        assert nq > 0.3 * cam["width"] * cam["height"]


def test_env_render_matches_oracle(env):
    api, ctx, vol, orc, params, cam, dirs, irr = env
    got = ctx.render_env(vol, cam, dirs, irr, precision=api.F32).cpu().numpy().ravel().astype(np.float64)
    ctx.sync_status()
    ref = orc.render_pixels_env(cam, np.arange(got.size), dirs.astype(np.float64), irr.astype(np.float64),
                                params=params.astype(np.float64))
    tol = 1e-3 * np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max()) + 1e-7
    frac = (np.abs(got - ref) <= tol).mean()
    assert frac >= 0.97, frac


def test_env_render_errors(env):
    api, ctx, vol, _, _, cam, dirs, irr = env
    with pytest.raises(api.RPNNError):
        ctx.render_env(vol, cam, dirs[:0], irr[:0])
    with pytest.raises(api.RPNNError):
        ctx.render_env(vol, cam, dirs * 2.0, irr)
    with pytest.raises(api.RPNNError):
        ctx.render_env(vol, cam, dirs, -irr)
    with pytest.raises(api.RPNNError):
        ctx.render_env(vol, cam, dirs, irr, mode=api.MODE_PATH)
