"""The cloud droplets' Lorenz-Mie phase function (Sec. 3.1) on the GPU, full and chopped
(full at a path's first bounce, the chopped function in the thinner medium after it):
renders (next-event estimation with the tabulated function, and path tracing that samples
it) and training records against the FP64 oracle with the same tables; switching the option
back restores the Henyey-Greenstein render exactly."""
import math

import numpy as np
import pytest

import oracle
from paper_1709_05418_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = ["PHASE_LORENZ_MIE", "PHASE_LORENZ_MIE_CHOPPED"]


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_05418_gb300 import api
    ctx = api.Context()
    dens = W.blob_cloud(64, seed=1)
    vol = ctx.load_volume(torch.from_numpy(dens).cuda())
    ctx.build_mips(vol)
    params = W.he_init(seed=2)
    ctx.set_weights(torch.from_numpy(params).cuda())
    orc = oracle.Volume(dens)
    cam = W.camera(dens.shape, 48, 40, spp=1, seed=3, light_seed=4)
    yield api, ctx, vol, orc, params, cam
    ctx.close()


def _close_frac(got, ref):
    tol = 1e-3 * np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max()) + 1e-7
    return (np.abs(got - ref) <= tol).mean()


def _render(api, ctx, vol, cam, kind, mode, precision=None):
    ctx.set_phase_function(vol, kind)
    try:
        img = ctx.render(vol, cam, precision=precision or api.F32, mode=mode)
        ctx.sync_status()
    finally:
        ctx.set_phase_function(vol, api.PHASE_HG)
    return img.cpu().numpy().ravel().astype(np.float64)


def _oracle_render(orc, kind, cam, n, params=None, mode=0):
    orc.set_phase(kind)
    try:
        return orc.render_pixels(cam, np.arange(n), params=params, mode=mode)
    finally:
        orc.set_phase(0)


@pytest.mark.parametrize("kind", KINDS)
def test_lorenz_mie_single_scatter_render_matches_oracle(env, kind):
    """Single scattering: next-event estimation evaluates the full table at the camera's
    vertex, through the chopped medium's thinner volume where it is chopped."""
    api, ctx, vol, orc, _, cam = env
    k = getattr(api, kind)
    hg = _render(api, ctx, vol, cam, api.PHASE_HG, api.MODE_SINGLE)
    got = _render(api, ctx, vol, cam, k, api.MODE_SINGLE)
    ref = _oracle_render(orc, k, cam, got.size, mode=0)
    # where light reaches the camera the HG render is far from the Lorenz-Mie one
    lit = ref > 0
    assert lit.mean() > 0.2
    assert _close_frac(hg[lit], ref[lit]) < 0.5
    assert _close_frac(got, ref) >= 0.97, _close_frac(got, ref)
    # switching back restores the HG render exactly
    assert np.array_equal(_render(api, ctx, vol, cam, api.PHASE_HG, api.MODE_SINGLE), hg)


@pytest.mark.parametrize("kind", KINDS)
def test_lorenz_mie_path_render_matches_oracle(env, kind):
    """Path tracing: every bounce samples its direction from the table and evaluates it for
    next-event estimation; the paths follow the oracle's decision by decision."""
    api, ctx, vol, orc, _, cam = env
    k = getattr(api, kind)
    hg = _render(api, ctx, vol, cam, api.PHASE_HG, api.MODE_PATH)
    got = _render(api, ctx, vol, cam, k, api.MODE_PATH)
    ref = _oracle_render(orc, k, cam, got.size, mode=1)
    lit = ref > 0
    assert _close_frac(hg[lit], ref[lit]) < 0.5
    frac = _close_frac(got, ref)
    print(f"{kind} path render: {frac:.4f} of pixels within 1e-3 of the oracle")
    assert frac >= 0.9, frac
    assert abs(got.mean() / ref.mean() - 1) <= 0.02


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("precision", ["F32", "BF16"])
def test_lorenz_mie_direct_term_of_rpnn_render(env, kind, precision):
    """RPNN render: only the direct (next-event) term at the shading point sees the phase
    function, the network output is the same, so the change from HG to Lorenz-Mie is the
    change of that term, and it matches the oracle's change."""
    api, ctx, vol, orc, params, cam = env
    k = getattr(api, kind)
    prec = getattr(api, precision)
    p64 = params.astype(np.float64)
    n = cam["width"] * cam["height"]
    hg = _render(api, ctx, vol, cam, api.PHASE_HG, api.MODE_RPNN, precision=prec)
    got = _render(api, ctx, vol, cam, k, api.MODE_RPNN, precision=prec)
    ref_hg = _oracle_render(orc, 0, cam, n, params=p64)
    ref = _oracle_render(orc, k, cam, n, params=p64)
    d_got, d_ref = got - hg, ref - ref_hg
    assert np.linalg.norm(d_ref) > 0
    # the network output is far larger than the direct term: the FP32 sums leave the change
    # to a few per cent per pixel
    rel = np.linalg.norm(d_got - d_ref) / np.linalg.norm(d_ref)
    assert rel <= 0.1, rel


@pytest.mark.parametrize("kind", KINDS)
def test_lorenz_mie_records_match_oracle(env, kind):
    api, ctx, vol, orc, _, _ = env
    k = getattr(api, kind)
    n = 48
    ctx.set_phase_function(vol, k)
    try:
        x, d, wl, lab, npaths = [t.cpu().numpy() for t in
                                 ctx.gen_records(vol, 0, n, 77, rel_ci=0.1, n_min=32, n_max=2048)]
        ctx.sync_status()
    finally:
        ctx.set_phase_function(vol, api.PHASE_HG)
    orc.set_phase(k)
    ok_lab = 0
    try:
        for i in range(n):
            r = orc.gen_record(77, i, rel_ci=0.1, n_min=32, n_max=2048)
            assert np.abs(wl[i] - r["wl"]).max() < 1e-5
            hw = max(r["half_width"], 1e-6) if math.isfinite(r["half_width"]) else r["label"]
            if abs(lab[i] - r["label"]) <= 3 * hw + 1e-6:
                ok_lab += 1
    finally:
        orc.set_phase(0)
    assert ok_lab >= 0.9 * n
    assert np.all(npaths >= 32) and np.all(npaths <= 2048)


def test_phase_function_errors(env):
    api, ctx, vol, _, _, _ = env
    with pytest.raises(api.RPNNError):
        ctx.set_phase_function(vol, 3)
    with pytest.raises(api.RPNNError):
        ctx.set_phase_function(12345, api.PHASE_LORENZ_MIE)
