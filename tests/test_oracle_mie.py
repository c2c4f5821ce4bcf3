"""Pins for the oracle's Lorenz-Mie phase function (Sec. 3.1; Bohren & Huffman's series):
the Rayleigh limit, energy conservation without absorption, the extinction paradox for
large spheres, and the tabulated cloud phase function's normalisation, sampling table and
asymmetry."""
import math

import numpy as np
import pytest


def test_small_spheres_scatter_like_a_dipole(orc):
    mu = np.linspace(-1.0, 1.0, 41)
    s11, qe, qs = orc.mie_single(1e-2, 1.33, 0.0, mu)
    assert np.allclose(s11 / s11[-1], 0.5 * (1.0 + mu * mu), rtol=1e-4)
    # Rayleigh efficiency 8/3 x^4 |(m^2-1)/(m^2+2)|^2
    m2 = 1.33 ** 2
    ray = 8.0 / 3.0 * 1e-8 * ((m2 - 1.0) / (m2 + 2.0)) ** 2
    assert abs(qs - ray) <= 1e-3 * ray


def test_no_absorption_conserves_energy_and_large_spheres_extinguish_twice(orc):
    mu = np.linspace(-1.0, 1.0, 5)
    for x in (0.5, 3.0, 25.0, 180.0):
        _, qe, qs = orc.mie_single(x, 1.333, 0.0, mu)
        assert abs(qe - qs) <= 1e-9 * qe, (x, qe, qs)
    _, qe, _ = orc.mie_single(600.0, 1.333, 0.0, mu)
    assert abs(qe - 2.0) < 0.05, qe
    # absorption removes energy: Q_ext > Q_sca
    _, qe, qs = orc.mie_single(10.0, 1.333, 0.05, mu)
    assert qe > qs * 1.05


@pytest.mark.parametrize("x,m_im", [(0.5, 0.0), (3.0, 0.0), (25.0, 0.0), (10.0, 0.05)])
def test_angular_intensity_integrates_to_the_scattering_efficiency(orc, x, m_im):
    """Q_sca from the coefficient series (sum of (2n+1)(|a_n|^2 + |b_n|^2)) equals the
    integral of the angular intensity, (2 / x^2) int_{-1}^{1} (|S1|^2 + |S2|^2)/2 dmu, which
    runs through the angular functions pi_n, tau_n instead (Bohren & Huffman's Eq. 4.61 and
    the definition of the scattering cross section)."""
    mu, w = np.polynomial.legendre.leggauss(1500)
    s11, _, qs = orc.mie_single(x, 1.333, m_im, mu)
    q_int = 2.0 / (x * x) * float((w * s11).sum())
    assert abs(q_int - qs) <= 1e-9 * qs, (q_int, qs)


def test_cloud_phase_table(orc):
    p, cdf, ce = orc.lm_table()
    assert p.size == orc.LM_BINS and np.all(p > 0)
    dom = 2.0 * math.pi * (ce[:-1] - ce[1:])
    assert abs((p * dom).sum() - 1.0) < 1e-12
    assert np.allclose(np.diff(cdf), p * dom, rtol=1e-12, atol=1e-13) and cdf[0] == 0 and cdf[-1] == 1.0
    assert np.allclose(ce, np.cos(np.arange(orc.LM_BINS + 1) * math.pi / orc.LM_BINS), atol=1e-15)
    # strongly forward-peaked cloud droplets: asymmetry parameter about 0.85-0.87
    mid = 0.5 * (ce[:-1] + ce[1:])
    g = (p * dom * mid).sum()
    assert 0.82 < g < 0.9, g
    assert p[0] / p[900] > 1e3          # forward peak against 90 degrees
    assert p[-1] > p[1400]              # the glory / back-scattering rise


def test_chopped_table(orc):
    """The chopped table (Sec. 3.1): the peak below 5 degrees removed, the rest renormalised;
    the removed fraction is about half the scattered light, as the extinction paradox gives
    for droplets much larger than the wavelength (diffraction carries half the extinction)."""
    from paper_1709_05418_gb300 import workloads as W
    p, cdf, ce = orc.lm_table()
    vol = orc.Volume(W.blob_cloud(16, seed=1), 0.9, 0.85)
    vol.set_phase(2)
    f, scale, alb_c = vol.chop_params()
    pc, cdfc = vol.lm_chopped_table()
    k = orc.LM_CHOP_BINS
    assert abs(math.degrees(math.acos(ce[k])) - 5.0) < 1e-9
    dom = 2.0 * math.pi * (ce[:-1] - ce[1:])
    assert abs(f - (p[:k] * dom[:k]).sum()) < 1e-12
    assert 0.35 < f < 0.55, f
    assert np.all(pc[:k] == 0) and np.allclose(pc[k:], p[k:] / (1.0 - f), rtol=1e-12)
    assert abs((pc * dom).sum() - 1.0) < 1e-12 and cdfc[-1] == 1.0
    assert np.all(cdfc[:k + 1] == 0) and np.allclose(np.diff(cdfc), pc * dom, rtol=1e-12, atol=1e-13)
    # the asymmetry splits into the peak's and the chopped function's
    mid = 0.5 * (ce[:-1] + ce[1:])
    g, g_c = (p * dom * mid).sum(), (pc * dom * mid).sum()
    g_peak = (p[:k] * dom[:k] * mid[:k]).sum() / f
    assert abs(g - (f * g_peak + (1.0 - f) * g_c)) < 1e-12 and g_peak > math.cos(math.radians(5.0))
    # chopping moves light from scattering to "not scattered": the absorption coefficient
    # (1 - albedo) mu_t is kept and the scattering coefficient drops by the factor 1 - f
    assert abs((1.0 - alb_c) * scale - (1.0 - 0.9)) < 1e-14
    assert abs(alb_c * scale - (1.0 - f) * 0.9) < 1e-14
    # without absorption the chopped medium does not absorb either
    vol1 = orc.Volume(W.blob_cloud(16, seed=1), 1.0, 0.85)
    vol1.set_phase(2)
    assert vol1.chop_params()[2] == 1.0
    vol.close()
    vol1.close()


def test_scaled_tracking_is_beer_lambert_of_the_thinner_medium(orc):
    """The chopped medium's transport (extinction s mu_t) against closed forms on the
    constant cube: ratio-tracking mean exp(-s tau), delta-tracking free paths 1 - exp(-s tau)."""
    from scipy import integrate, stats
    n, mu0, s = 8, 1.5, 0.55
    ramp = lambda u: np.clip(np.minimum(u + 1.0, n - u), 0.0, 1.0)
    tau = lambda x0, x1: integrate.quad(lambda x: mu0 * ramp(x * n - 0.5), x0, x1,
                                        points=[0.5 / n, 1 - 0.5 / n], limit=200)[0]
    v = orc.Volume(np.full((n, n, n), mu0, np.float32), 0.9, 0.85)
    o = np.array([-0.5, 3.5 / n, 3.5 / n])
    d = np.array([1.0, 0.0, 0.0])
    T = np.array([v.ratio_track(o, d, 77, i, 0, scale=s) for i in range(4000)])
    exact = math.exp(-s * tau(0.0, 1.0))
    assert abs(T.mean() - exact) < 4 * T.std() / math.sqrt(T.size)
    # s = 1 is the unscaled estimator, draw for draw
    assert all(v.ratio_track(o, d, 77, i, 0, scale=1.0) == v.ratio_track(o, d, 77, i, 0) for i in range(50))
    o = np.array([-0.25, 4.5 / n, 4.5 / n])
    hits, xs, m = 0, [], 4000
    for i in range(m):
        r, x, _ = v.delta_track(o, d, 99, i, 0, scale=s)
        if r == 1:
            hits += 1
            xs.append(x[0])
    p = 1 - math.exp(-s * tau(0.0, 1.0))
    assert abs(hits / m - p) < 4 * math.sqrt(p * (1 - p) / m)
    grid = np.linspace(0, 1, 401)
    taus = np.array([tau(0.0, x) if x > 0 else 0.0 for x in grid])
    F = lambda x: np.interp(x, grid, (1 - np.exp(-s * taus)) / p)
    assert stats.kstest(xs, F).pvalue > 1e-3
    v.close()


@pytest.mark.parametrize("kind", [1, 2])
def test_lorenz_mie_single_scattering_matches_quadrature(orc, kind):
    """Single scattering of a slab pixel with the table: the camera's vertex scatters with the
    full Lorenz-Mie function (the first bounce) in both modes; in the chopped mode the light
    reaches it through the thinner medium (extinction s mu_t)."""
    from scipy import integrate
    n, mu0, alb = 8, 1.5, 0.8
    ramp = lambda u: float(np.clip(min(u + 1.0, n - u), 0.0, 1.0))
    v = orc.Volume(np.full((n, n, n), mu0, np.float32), alb, 0.85)
    v.set_phase(kind)
    s = v.chop_params()[1]
    assert (s == 1.0) == (kind == 1)
    y0, z0 = 3.5 / n, 4.5 / n
    a = math.radians(23.456)                    # scattering angle 113.456 degrees: inside a bin
    wl = np.array([-math.sin(a), math.cos(a), 0.0])
    cam = {"cam_pos": [-1.0, y0, z0], "cam_fwd": [1.0, 0, 0], "cam_right": [0, 0, -1.0],
           "cam_up": [0, 1.0, 0], "tan_half_fov_y": 1e-9, "width": 64, "height": 64,
           "spp": 8, "seed": 4242, "light_dir": wl, "light_E": 1.0}
    px = v.render_pixels(cam, np.arange(64 * 64), params=None, mode=0)
    p_tab = orc.lm_table()[0]
    theta = math.acos(float(np.dot([1.0, 0.0, 0.0], wl)))
    ph = p_tab[int(math.degrees(theta) / 0.1)]

    def tau_light(x):
        s_end = min(x / math.sin(a), (1.0 - y0) / math.cos(a))      # leaves the unit box
        fx = lambda u: mu0 * ramp((x - u * math.sin(a)) * n - 0.5) * ramp((y0 + u * math.cos(a)) * n - 0.5)
        return integrate.quad(fx, 0.0, s_end, limit=200)[0]

    def tau_cam(x):
        return integrate.quad(lambda u: mu0 * ramp(u * n - 0.5), 0.0, x, points=[0.5 / n], limit=200)[0]

    def f(x):
        return mu0 * ramp(x * n - 0.5) * math.exp(-tau_cam(x)) * ph * math.exp(-s * tau_light(x))

    exp = alb * integrate.quad(f, 0, 1, points=[0.5 / n, 1 - 0.5 / n], limit=100)[0]
    se = px.std() / math.sqrt(px.size)
    assert abs(px.mean() - exp) < 4 * se + 1e-9, (px.mean(), exp, se)
    v.close()


def test_chopping_nothing_is_the_full_function(orc):
    """Chopped mode with no bins removed follows the full Lorenz-Mie paths exactly."""
    from paper_1709_05418_gb300 import workloads as W
    dens = W.blob_cloud(32, seed=1)
    a, b = orc.Volume(dens), orc.Volume(dens)
    a.set_phase(1)
    b.set_phase(2, chop_bins=0)
    assert b.chop_params() == (0.0, 1.0, a.chop_params()[2])
    cam = W.camera(dens.shape, 16, 12, spp=1, seed=3, light_seed=4)
    pix = np.arange(16 * 12)
    assert np.array_equal(a.render_pixels(cam, pix, mode=1), b.render_pixels(cam, pix, mode=1))
    for r in range(4):
        ra, rb = a.gen_record(7, r, 0.1, 32, 256), b.gen_record(7, r, 0.1, 32, 256)
        assert ra["label"] == rb["label"] and ra["npaths"] == rb["npaths"]
    a.close()
    b.close()


def test_chopped_lorenz_mie_approximates_the_full_function(orc):
    """Sec. 3.1: the chopped function (after the first bounce, in the thinner medium) gives
    nearly the full function's in-scattered radiance at far lower estimator variance."""
    from paper_1709_05418_gb300 import workloads as W
    v = orc.Volume(W.blob_cloud(64, seed=1))
    full, chop = [], []
    for rec in range(6):
        r = v.gen_record(5, rec, rel_ci=0.1, n_min=32, n_max=256)
        for kind, out in ((1, full), (2, chop)):
            v.set_phase(kind)
            st, mean, var = v.estimate_Li(9, rec, r["x"], r["d"], r["wl"], 20000)
            assert st == 0
            out.append((mean, var))
        v.set_phase(0)
    mf, vf = np.array(full).T
    mc, vc = np.array(chop).T
    se = np.sqrt((vf + vc) / 20000)
    print("full", mf, "chopped", mc, "se", se)
    assert abs(mc.sum() - mf.sum()) <= 4 * np.sqrt((se ** 2).sum()) + 0.05 * mf.sum()
    assert vc.sum() < 0.2 * vf.sum()
    v.close()


def test_chopped_first_collision_term_matches_quadrature(orc):
    """The first-collision part of L_i in the chopped mode against brute-force quadrature on
    the constant cube: the new direction d' from the full table at x (the first bounce), the
    collision density s mu e^(-s tau) of the thinner medium, survival with the chopped
    albedo, and next-event estimation with the chopped table through the thinner medium:
        alb_c int p(d.d') int_0^b s mu(t) e^(-s tau(t)) p_c(d'.wl) e^(-s tau_l(t)) dt dd'.
    With the tracing direction d equal to the light direction both tables are functions of
    the same angle, so the sphere integral runs bin by bin over the tables (exact for these
    piecewise-constant functions) with the smooth transport factor at 0.5-degree nodes."""
    n, mu0, alb = 8, 1.5, 0.8
    ramp = lambda u: np.clip(np.minimum(u + 1.0, n - u), 0.0, 1.0)

    def mu(pt):
        u = pt * n - 0.5
        return mu0 * ramp(u[..., 0]) * ramp(u[..., 1]) * ramp(u[..., 2])

    def exit_dist(pt, d):
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = np.where(d > 0, (1.0 - pt) / d, np.where(d < 0, -pt / d, np.inf))
        return t1.min(axis=-1)

    def transport(x, dirs, wl, s, ns=160, nl=80):
        b = exit_dist(np.broadcast_to(x, dirs.shape), dirs)
        dt = (b / ns)[:, None]
        pts = x[None, None, :] + (b[:, None] * (np.arange(ns) + 0.5) / ns)[..., None] * dirs[:, None, :]
        m = s * mu(pts)
        tau = np.cumsum(m * dt, axis=1) - 0.5 * m * dt
        bl = exit_dist(pts, np.broadcast_to(wl, pts.shape))
        lp = pts[..., None, :] + (bl[..., None] * (np.arange(nl) + 0.5) / nl)[..., None] * wl
        tau_l = s * mu(lp).sum(-1) * bl / nl
        return (m * np.exp(-tau - tau_l) * dt).sum(1)

    v = orc.Volume(np.full((n, n, n), mu0, np.float32), alb, 0.85)
    v.set_phase(2)
    _, s, alb_c = v.chop_params()
    p, _, ce = orc.lm_table()
    pc, _ = v.lm_chopped_table()
    x = np.array([0.5, 0.45, 0.55])
    wl = np.array([1.0, 1.0, 0.3]) / np.linalg.norm([1.0, 1.0, 0.3])
    b1 = np.cross(wl, [0.0, 0.0, 1.0])
    b1 /= np.linalg.norm(b1)
    b2 = np.cross(wl, b1)
    nodes = np.linspace(math.radians(orc.LM_CHOP_BINS * 0.1), math.pi, 351)
    phis = (np.arange(12) + 0.5) * 2.0 * math.pi / 12
    vals = [transport(x, math.cos(th) * wl[None, :] + math.sin(th) * (np.cos(phis)[:, None] * b1 +
                                                                         np.sin(phis)[:, None] * b2), wl, s).mean()
            for th in nodes]
    mid = (np.arange(orc.LM_BINS) + 0.5) * math.pi / orc.LM_BINS
    dom = 2.0 * math.pi * (ce[:-1] - ce[1:])
    exp = alb_c * float((p * pc * dom * np.interp(mid, nodes, vals)).sum())
    npaths = 400000
    r, mean, var = v.estimate_Li(321, 0, x, wl, wl, npaths, max_bounces=1)
    se = math.sqrt(var / npaths)
    assert r == 0
    assert abs(mean - exp) < 4 * se + 0.005 * exp, (mean, exp, se)
    v.close()
