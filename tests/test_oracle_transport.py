"""Pins for the oracle's Monte Carlo transport: Henyey-Greenstein phase function,
delta tracking, ratio tracking and single scattering (Sec. 3.2 Eq. 1, Sec. 4.4)."""
import math

import numpy as np
from scipy import integrate, stats

N, MU0 = 8, 1.5          # constant 8^3 cube, extinction 1.5 per unit


def ramp(u):
    """1-D profile of the trilinear field of a constant grid (voxel centres at integer
    u, zero outside): rises over [-1, 0], flat on [0, n-1], falls over [n-1, n]."""
    return np.clip(np.minimum(u + 1.0, N - u), 0.0, 1.0)


def tau_axis(x0, x1):
    """optical depth between world x0 < x1 along an axis through interior voxel centres"""
    f = lambda x: MU0 * ramp(x * N - 0.5)
    return integrate.quad(f, x0, x1, points=[0.5 / N, 1 - 0.5 / N], limit=200)[0]


def cube(orc, albedo=0.99, g=0.85):
    return orc.Volume(np.full((N, N, N), MU0, np.float32), albedo, g)


def test_hg_normalised_and_mean_cosine(orc):
    for g in (0.0, 0.3, 0.85, -0.5):
        norm = integrate.quad(lambda m: 2 * math.pi * orc.hg(g, m), -1, 1, limit=200)[0]
        mc = integrate.quad(lambda m: 2 * math.pi * m * orc.hg(g, m), -1, 1, limit=200)[0]
        assert abs(norm - 1.0) < 1e-8 and abs(mc - g) < 1e-8


def test_hg_sampling_distribution(orc):
    g = 0.85
    rng = np.random.default_rng(5)
    d = np.array([0.2, -0.5, 0.7])
    d /= np.linalg.norm(d)
    cos, phi_ok = [], []
    for _ in range(4000):
        o = orc.sample_hg(g, d, rng.random(), rng.random())
        assert abs(np.linalg.norm(o) - 1) < 1e-12
        cos.append(np.dot(o, d))
    cdf = lambda m: (1 - g * g) / (2 * g) * ((1 + g * g - 2 * g * np.asarray(m)) ** -0.5 - 1 / (1 + g))
    assert stats.kstest(cos, cdf).pvalue > 1e-3


def test_ratio_tracking_mean_is_beer_lambert(orc):
    v = cube(orc)
    y0 = z0 = 3.5 / N
    o = np.array([-0.5, y0, z0])
    d = np.array([1.0, 0.0, 0.0])
    T = np.array([v.ratio_track(o, d, 77, i, 0) for i in range(4000)])
    exact = math.exp(-MU0 * (N - 0.25) / N)
    assert abs(math.exp(-tau_axis(0, 1)) - exact) < 1e-12
    assert abs(T.mean() - exact) < 4 * T.std() / math.sqrt(T.size)
    assert np.all(T >= 0) and np.all(T <= 1)


def test_delta_tracking_free_path_distribution(orc):
    v = cube(orc)
    y0 = z0 = 4.5 / N
    o = np.array([-0.25, y0, z0])
    d = np.array([1.0, 0.0, 0.0])
    hits, xs = 0, []
    n = 4000
    for i in range(n):
        r, x, t = v.delta_track(o, d, 99, i, 0)
        if r == 1:
            hits += 1
            xs.append(x[0])
            assert abs(t - (x[0] + 0.25)) < 1e-12
    tau1 = tau_axis(0, 1)
    p = 1 - math.exp(-tau1)
    assert abs(hits / n - p) < 4 * math.sqrt(p * (1 - p) / n)
    grid = np.linspace(0, 1, 401)
    taus = np.array([tau_axis(0, x) if x > 0 else 0.0 for x in grid])
    F = lambda x: np.interp(x, grid, (1 - np.exp(-taus)) / p)
    assert stats.kstest(xs, F).pvalue > 1e-3


def test_single_scattering_pixel_matches_quadrature(orc):
    g, alb = 0.6, 0.8
    v = cube(orc, alb, g)
    y0, z0 = 3.5 / N, 4.5 / N
    wl = np.array([0.0, 1.0, 0.0])
    cam = {"cam_pos": [-1.0, y0, z0], "cam_fwd": [1.0, 0, 0], "cam_right": [0, 0, -1.0],
           "cam_up": [0, 1.0, 0], "tan_half_fov_y": 1e-9, "width": 64, "height": 64,
           "spp": 8, "seed": 4242, "light_dir": wl, "light_E": 1.0}
    px = v.render_pixels(cam, np.arange(64 * 64), params=None, mode=0)
    # expectation: alb * int mu(s) T_cam(s) p(d.wl) T_light(s) ds along the pixel ray
    ty = integrate.quad(lambda y: ramp(y * N - 0.5), y0, 1.0, points=[1 - 0.5 / N])[0] * MU0

    def f(x):
        rx = ramp(x * N - 0.5)
        return MU0 * rx * math.exp(-tau_axis(0, x)) * orc.hg(g, 0.0) * math.exp(-rx * ty)

    exp = alb * integrate.quad(f, 0, 1, points=[0.5 / N, 1 - 0.5 / N], limit=200)[0]
    se = px.std() / math.sqrt(px.size)
    assert abs(px.mean() - exp) < 4 * se + 1e-9, (px.mean(), exp, se)
    # plain path tracing adds the (non-negative) indirect part
    pt = v.render_pixels(cam, np.arange(64 * 64), params=None, mode=1)
    assert pt.mean() > px.mean()


def test_primary_sample_is_consistent(orc):
    v = cube(orc)
    cam = {"cam_pos": [0.5, 0.5, -1.5], "cam_fwd": [0, 0, 1.0], "cam_right": [1.0, 0, 0],
           "cam_up": [0, 1.0, 0], "tan_half_fov_y": 0.2, "width": 16, "height": 16,
           "spp": 1, "seed": 9, "light_dir": [0.0, 0.6, 0.8], "light_E": 2.0}
    pix = v.render_pixels(cam, np.arange(256), params=None, mode=0)
    for p in range(0, 256, 17):
        hit, x, d, Ld = v.primary(cam, p, 0)
        if hit == 1:
            assert abs(np.linalg.norm(d) - 1) < 1e-12
            assert np.all(x >= 0) and np.all(x <= 1)
            assert v.density(x) > 0
            assert abs(pix[p] - 0.99 * Ld) < 1e-15
            # the shadow ray estimate is bounded by E * p(d . wl)
            assert 0 <= Ld <= 2.0 * orc.hg(0.85, float(np.dot(d, cam["light_dir"]))) + 1e-15
        else:
            assert pix[p] == 0.0


def test_environment_render_is_the_superposition_of_its_lights(orc):
    """Sec. 4.4's environment emitter as directional samples: one light reproduces the
    single-light render, a light split into two halves of its irradiance gives the same
    image, and the image is linear in the irradiances (single scattering and a network
    prediction alike scale with E)."""
    from paper_1709_05418_gb300 import workloads as W
    vol = orc.Volume(W.blob_cloud(24, nblobs=4, seed=3))
    cam = W.camera((24, 24, 24), 12, 10, spp=2, seed=8, light_seed=9)
    params = W.he_init(seed=2, K_=10).astype(np.float64)
    pix = np.arange(120)
    w0 = np.asarray(cam["light_dir"], np.float64)
    w1 = np.array([0.0, 0.6, 0.8])
    single = vol.render_pixels(cam, pix, params=params)
    assert np.count_nonzero(single) > 20
    one = vol.render_pixels_env(cam, pix, [w0], [1.0], params=params)
    assert np.array_equal(one, single)
    halves = vol.render_pixels_env(cam, pix, [w0, w0], [0.5, 0.5], params=params)
    assert np.allclose(halves, single, rtol=1e-12, atol=1e-15)
    a = vol.render_pixels_env(cam, pix, [w0, w1], [1.0, 2.0], params=params)
    b = vol.render_pixels_env(cam, pix, [w0, w1], [3.0, 6.0], params=params)
    assert np.allclose(b, 3.0 * a, rtol=1e-12, atol=1e-15)
    second = vol.render_pixels(dict(cam, light_dir=tuple(w1), light_E=2.0), pix, params=params)
    assert np.allclose(a, single + second, rtol=1e-12, atol=1e-15)
    assert not np.allclose(a, single)
    vol.close()


def _sparse_grid(n=20, seed=5):
    """Heterogeneous grid with empty bricks: random values in two blobs, zero elsewhere."""
    rng = np.random.default_rng(seed)
    g = np.zeros((n, n, n), np.float32)
    g[2:9, 3:12, 1:10] = rng.uniform(5.0, 40.0, size=(7, 9, 9))
    g[12:19, 10:18, 11:19] = rng.uniform(0.0, 8.0, size=(7, 8, 8))
    return g


def test_brick_majorants_are_the_max_of_the_interpolated_voxels(orc):
    g = _sparse_grid()
    vol = orc.Volume(g)
    bm = vol.brick_majorants()
    n = g.shape[0]
    pad = np.zeros((n + 2, n + 2, n + 2), np.float32)
    pad[1:-1, 1:-1, 1:-1] = g                       # voxel i at pad index i + 1
    for bz in range(bm.shape[0]):
        for by in range(bm.shape[1]):
            for bx in range(bm.shape[2]):
                sl = pad[8 * bz:8 * bz + 10, 8 * by:8 * by + 10, 8 * bx:8 * bx + 10]
                assert bm[bz, by, bx] == sl.max()
    assert (bm == 0).any() and (bm > 0).any()
    # every point's trilinear density stays below its brick's majorant
    rng = np.random.default_rng(1)
    ext = n / n
    for p in rng.uniform(0.0, ext, size=(3000, 3)):
        b = np.minimum((p * n / 8).astype(int), np.array(bm.shape[::-1]) - 1)
        assert vol.density(p) <= bm[b[2], b[1], b[0]] + 1e-12
    vol.close()


def test_brick_tracking_matches_global_majorant_in_distribution(orc):
    """On a grid with empty and dense bricks, free-flight distances of the brick-majorant
    delta tracking and of the global-majorant one follow the same law (two-sample KS), and
    ratio tracking's mean transmittance matches exp(-optical depth) by fine ray marching."""
    g = _sparse_grid()
    vol = orc.Volume(g)
    o = np.array([-0.2, 0.25, 0.22])
    d = np.array([1.0, 0.12, 0.2]); d /= np.linalg.norm(d)
    def dists(glob):
        out = []
        for s in range(3000):
            r, x, t = vol.delta_track(o, d, 1234, s, 0, global_majorant=glob)
            out.append(t if r == 1 else 10.0)
        return np.array(out)
    a, b = dists(False), dists(True)
    assert (a < 10).mean() > 0.3
    assert stats.ks_2samp(a, b).pvalue > 1e-3
    ts = np.linspace(0.0, 2.0, 200001)
    mus = np.array([vol.density(o + t * d) for t in ts[::20]])
    tau = np.trapezoid(mus, ts[::20])
    T = np.array([vol.ratio_track(o, d, 99, s, 0) for s in range(4000)])
    assert abs(T.mean() - math.exp(-tau)) <= 4 * T.std() / math.sqrt(T.size) + 1e-4
    vol.close()


def test_furnace(orc):
    """Energy conservation of the whole transport (the furnace test): a non-absorbing cube
    (albedo 1) under a uniform environment of unit radiance -- here 200 directional lights
    on a Fibonacci sphere, each of irradiance 4 pi / 200 (Sec. 4.4's environment as
    directional samples) -- has unit radiance everywhere inside, so at every collision the
    direct plus path-traced in-scattering add up to 1 on average, and a pixel whose ray meets
    the medium with probability 1 - exp(-tau) sees that fraction of it."""
    v = cube(orc, 1.0, 0.3)
    y0, z0 = 3.5 / N, 4.5 / N
    K = 200
    i = np.arange(K) + 0.5
    zc = 1 - 2 * i / K
    ph = math.pi * (1 + 5 ** 0.5) * i
    r = np.sqrt(1 - zc * zc)
    dirs = np.stack([r * np.cos(ph), r * np.sin(ph), zc], 1)
    W_, H_, spp = 32, 32, 8
    cam = {"cam_pos": [-1.0, y0, z0], "cam_fwd": [1.0, 0, 0], "cam_right": [0, 0, -1.0],
           "cam_up": [0, 1.0, 0], "tan_half_fov_y": 1e-9, "width": W_, "height": H_,
           "spp": spp, "seed": 77, "light_dir": dirs[0], "light_E": 1.0}
    pix = np.arange(W_ * H_)
    irr = np.full(K, 4 * math.pi / K)
    px = v.render_pixels_env(cam, pix, dirs, irr, mode=1)
    hits = np.array([[v.primary(cam, int(p), s)[0] == 1 for s in range(spp)] for p in pix])
    # the visible-point fraction is Beer-Lambert's
    q = 1.0 - math.exp(-tau_axis(0, 1))
    assert abs(hits.mean() - q) < 4 * math.sqrt(q * (1 - q) / hits.size)
    # in-scattered radiance at the collisions: unit on average (pixel sums over hits only)
    per_hit = px * spp
    n_hit = hits.sum(1)
    mean = per_hit.sum() / n_hit.sum()
    # standard error from the per-pixel sums (ratio estimator)
    se = np.sqrt(((per_hit - mean * n_hit) ** 2).sum()) / n_hit.sum()
    assert abs(mean - 1.0) < 4 * se + 0.01, (mean, se)
    # single scattering alone falls well short of it
    ss = v.render_pixels_env(cam, pix, dirs, irr, mode=0) * spp
    assert ss.sum() / n_hit.sum() < 0.8
