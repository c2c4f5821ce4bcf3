"""FP8 (E4M3) form of the network (per-tensor scales, FP32 accumulation) against the FP64
oracle: the E4M3 descriptor is the round-to-nearest-even E4M3 value of the bit-exact FP32
descriptor; network outputs stay within the FP8 budget (relative L2 <= 3e-2 over a
batch, and per element within 9e-2 of max(|y|, median |y|)); rendered images are reported and held to 5e-2 (the network's error reaches them
through the share of each pixel that is the prediction); the FP8 path refuses to run
before calibration."""
import numpy as np
import pytest

import oracle
from paper_1709_05418_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP8_REL = 3e-2        # network output, relative L2 over the batch
# network output, per element: |err| <= FP8_ELEM * max(|y|, median |y|).  Three times the
# norm-wise bound, as the BF16 tests' per-element 3e-2 is three times their 1e-2: one E4M3
# rounding moves a value by up to 2^-4 = 6.25 %, and a prediction dominated by a few
# activations inherits about that (largest measured: 7.2e-2), so a per-element bound at the
# norm-wise 3e-2 is below the format's own resolution.
FP8_ELEM = 9e-2
FP8_IMG_REL = 5e-2    # rendered image, relative L2 over the pixels


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8_e4m3fn in this torch")
    from paper_1709_05418_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def ctx(api):
    c = api.Context()
    yield c
    c.close()


def cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


@pytest.fixture(scope="module")
def blob():
    return W.blob_cloud(64, seed=1)


@pytest.fixture(scope="module")
def blob_vol(ctx, blob):
    v = ctx.load_volume(cuda(blob))
    ctx.build_mips(v)
    return v


@pytest.fixture(scope="module")
def blob_orc(blob):
    return oracle.Volume(blob)


@pytest.fixture(scope="module")
def params():
    return W.he_init(seed=2)


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _queries(q, seed):
    x, d = W.random_queries((64, 64, 64), q, seed=seed, margin=0.2)
    wl = np.array([0.3, 0.5, -0.8])
    wl /= np.linalg.norm(wl)
    return x.astype(np.float32), d.astype(np.float32), wl.astype(np.float32)


def test_fp8_descriptor_is_e4m3_of_fp32(ctx, blob_vol):
    x, d, wl = _queries(257, seed=31)
    g32 = ctx.extract_descriptors(blob_vol, cuda(x), cuda(d), cuda(wl))
    g8 = ctx.extract_descriptors(blob_vol, cuda(x), cuda(d), cuda(wl), dtype=torch.uint8).cpu()
    assert g8.shape == (257, 10, 256)
    # the E4M3 rounding of the FP32 descriptor, taken on the CPU
    ref = g32.cpu().to(torch.float8_e4m3fn).view(torch.uint8)
    assert torch.equal(g8[:, :, :240], ref)
    assert int(g8[:, :, 240:].sum()) == 0


def test_fp8_requires_calibration(ctx, api, blob_vol, params):
    ctx.set_weights(cuda(params))
    cam = W.camera((64, 64, 64), 16, 16, seed=3, light_seed=4)
    with pytest.raises(api.RPNNError):
        ctx.render(blob_vol, cam, precision=api.FP8)
    z = torch.zeros((4, 10, 256), dtype=torch.uint8, device="cuda")
    with pytest.raises(api.RPNNError):
        ctx.mlp_forward(z, precision=api.FP8)


@pytest.mark.parametrize("q", [333, 152 * 128 * 2 + 77])
def test_fp8_mlp_within_budget(ctx, api, blob_vol, blob_orc, params, q, capsys):
    ctx.set_weights(cuda(params))
    # calibrate on other queries of the same cloud
    xc, dc, wlc = _queries(2048, seed=40)
    ctx.calibrate_fp8(ctx.extract_descriptors(blob_vol, cuda(xc), cuda(dc), cuda(wlc)))
    x, d, wl = _queries(333, seed=11)
    z32 = blob_orc.descriptor(x, d, wl, f32=True)                   # [333][10][226]
    ref = oracle.mlp_forward(params.astype(np.float64), z32.astype(np.float64))
    src = np.arange(q) % 333
    zp = np.zeros((333, 10, 256), np.float32)
    zp[:, :, :226] = z32
    z8 = torch.from_numpy(zp).to(torch.float8_e4m3fn).view(torch.uint8)[torch.from_numpy(src)].contiguous().cuda()
    g = ctx.mlp_forward(z8, precision=api.FP8).cpu().numpy().astype(np.float64)
    ctx.sync_status()
    assert np.all(np.isfinite(g))
    assert (ref > 0).mean() > 0.2
    err = _rel_l2(g, ref[src])
    r = ref[src]
    scale = np.maximum(np.abs(r), np.median(np.abs(r)))
    worst = float((np.abs(g - r) / scale).max())
    with capsys.disabled():
        print(f"\n[fp8] network vs FP64 oracle, {q} rows: rel L2 {err:.4f}, "
              f"largest |err| / max(|y|, median|y|) {worst:.4f}")
    assert err <= FP8_REL, err
    assert np.all(np.abs(g - r) <= FP8_ELEM * scale), worst


def test_fp8_render_within_budget(ctx, api, blob, blob_vol, blob_orc, params, capsys):
    ctx.set_weights(cuda(params))
    cam = W.camera(blob.shape, 64, 64, spp=1, seed=3, light_seed=4)
    hit, x, d, _ = ctx.trace_primary(blob_vol, cam)
    sel = hit.bool()
    wl = torch.as_tensor(np.asarray(cam["light_dir"], np.float32)).cuda()
    ctx.calibrate_fp8(ctx.extract_descriptors(blob_vol, x[sel].contiguous(), d[sel].contiguous(), wl))
    img = ctx.render(blob_vol, cam, precision=api.FP8)
    ctx.sync_status()
    got = img.cpu().numpy().ravel().astype(np.float64)
    ref = blob_orc.render_pixels(cam, np.arange(got.size), params=params.astype(np.float64))
    err = _rel_l2(got, ref)
    bf = ctx.render(blob_vol, cam, precision=api.BF16).cpu().numpy().ravel().astype(np.float64)
    with capsys.disabled():
        print(f"\n[fp8] image rel L2 vs FP64 oracle: FP8 {err:.4f}, BF16 {_rel_l2(bf, ref):.4f}")
    assert err <= FP8_IMG_REL, err


def test_networks_with_distinct_layer_biases(ctx, api, blob_vol, blob_orc):
    """Every layer with its own nonzero biases (trained networks have them; He
    initialisation sets them to zero): the E4M3 network, which adds each layer's FP32 bias
    in its epilogue, and the BF16 one, whose weight image carries them, stay within their
    budgets against the FP64 oracle."""
    params = W.he_init(seed=5)
    parts = W.split_params(params)
    rng = np.random.default_rng(6)
    flat, off = params.copy(), 0
    for name, arr in parts.items():
        if name.startswith("b"):
            flat[off:off + arr.size] = rng.normal(0.0, 0.05, size=arr.size)
        off += arr.size
    ctx.set_weights(cuda(flat))
    xc, dc, wlc = _queries(2048, seed=41)
    ctx.calibrate_fp8(ctx.extract_descriptors(blob_vol, cuda(xc), cuda(dc), cuda(wlc)))
    x, d, wl = _queries(333, seed=12)
    z32 = blob_orc.descriptor(x, d, wl, f32=True)
    ref = oracle.mlp_forward(flat.astype(np.float64), z32.astype(np.float64))
    assert (ref > 0).mean() > 0.2
    zp = np.zeros((333, 10, 256), np.float32)
    zp[:, :, :226] = z32
    z8 = torch.from_numpy(zp).to(torch.float8_e4m3fn).view(torch.uint8).cuda()
    g8 = ctx.mlp_forward(z8, precision=api.FP8).cpu().numpy().astype(np.float64)
    zb = torch.from_numpy(zp[:, :, :240].copy()).to(torch.bfloat16).cuda()
    g16 = ctx.mlp_forward(zb, precision=api.BF16).cpu().numpy().astype(np.float64)
    ctx.sync_status()
    scale = np.maximum(np.abs(ref), np.median(np.abs(ref)))
    assert _rel_l2(g8, ref) <= FP8_REL, _rel_l2(g8, ref)
    assert np.all(np.abs(g8 - ref) <= FP8_ELEM * scale)
    assert _rel_l2(g16, ref) <= 1e-2, _rel_l2(g16, ref)

