"""Pins for the oracle's training-record generator (Sec. 5.1) and its estimator of the
indirect in-scattered radiance L_i (Sec. 4)."""
import math

import numpy as np

from paper_1709_05418_gb300 import workloads as W

N, MU0 = 8, 1.5


def ramp(u):
    return np.clip(np.minimum(u + 1.0, N - u), 0.0, 1.0)


def mu(p):
    u = p * N - 0.5
    return MU0 * ramp(u[..., 0]) * ramp(u[..., 1]) * ramp(u[..., 2])


def exit_dist(p, d):
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = np.where(d > 0, (1.0 - p) / d, np.where(d < 0, -p / d, np.inf))
    return t1.min(axis=-1)


def hg(g, c):
    den = 1 + g * g - 2 * g * c
    return (1 - g * g) / (4 * math.pi * den ** 1.5)


def first_order_Li(x, d_in, wl, g, ndir=1500, ns=160, nl=80):
    """Brute-force quadrature of the single-collision term of L_i at x:
    int_S2 p(d_in.d') int_0^b mu T(x, x+s d') p(d'.wl) T_light ds dd'."""
    i = np.arange(ndir) + 0.5
    zc = 1 - 2 * i / ndir
    ph = math.pi * (1 + 5 ** 0.5) * i
    r = np.sqrt(1 - zc * zc)
    dirs = np.stack([r * np.cos(ph), r * np.sin(ph), zc], 1)
    b = exit_dist(np.broadcast_to(x, dirs.shape), dirs)
    frac = (np.arange(ns) + 0.5) / ns
    s = b[:, None] * frac[None, :]
    ds = (b / ns)[:, None]
    pts = x[None, None, :] + s[..., None] * dirs[:, None, :]
    m = mu(pts)
    tau = np.cumsum(m * ds, axis=1) - 0.5 * m * ds
    bl = exit_dist(pts, np.broadcast_to(wl, pts.shape))
    fl = (np.arange(nl) + 0.5) / nl
    lp = pts[..., None, :] + (bl[..., None] * fl)[..., None] * wl
    taul = mu(lp).sum(-1) * bl / nl
    inner = (m * np.exp(-tau) * np.exp(-taul) * ds).sum(1)
    w = hg(g, dirs @ d_in) * hg(g, dirs @ wl)
    return 4 * math.pi / ndir * (w * inner).sum()


def test_first_collision_term_matches_quadrature(orc):
    g = 0.3
    v = orc.Volume(np.full((N, N, N), MU0, np.float32), 1.0, g)
    x = np.array([0.5, 0.5, 0.5])
    d = np.array([0.0, 0.0, 1.0])
    wl = np.array([1.0, 1.0, 0.3])
    wl /= np.linalg.norm(wl)
    exp = first_order_Li(x, d, wl, g)
    r, mean, var = v.estimate_Li(123, 0, x, d, wl, 40000, max_bounces=1)
    se = math.sqrt(var / 40000)
    assert r == 0
    assert abs(mean - exp) < 4 * se + 0.01 * exp, (mean, exp, se)
    # with albedo 1/2 each collision survives with probability 1/2 (analog absorption)
    v2 = orc.Volume(np.full((N, N, N), MU0, np.float32), 0.5, g)
    _, m2, var2 = v2.estimate_Li(124, 0, x, d, wl, 40000, max_bounces=1)
    assert abs(m2 - 0.5 * exp) < 4 * math.sqrt(var2 / 40000) + 0.01 * exp
    # higher orders only add (non-negative) energy
    _, mall, _ = v.estimate_Li(123, 0, x, d, wl, 40000, max_bounces=0)
    assert mall > mean


def test_record_sampling(orc):
    dens = W.blob_cloud(24, seed=21)
    v = orc.Volume(dens, 0.9, 0.85)
    ds, wls = [], []
    for rec in range(64):
        r = v.gen_record(555, rec, rel_ci=0.2, n_min=16, n_max=512)
        assert r["status"] == 0
        x, d, wl = r["x"], r["d"], r["wl"]
        assert abs(np.linalg.norm(d) - 1) < 1e-12 and abs(np.linalg.norm(wl) - 1) < 1e-12
        assert np.all(x >= 0) and np.all(x <= 1) and v.density(x) > 0
        assert r["label"] >= 0 and 16 <= r["npaths"] <= 512
        if r["npaths"] < 512:
            assert r["half_width"] <= 0.2 * r["label"] + 1e-15
        ds.append(d)
        wls.append(wl)
    ds, wls = np.array(ds), np.array(wls)
    # uniform directions: mean ~ 0 (4 sigma = 4 / sqrt(3 * 64))
    assert np.all(np.abs(ds.mean(0)) < 0.3) and np.all(np.abs(wls.mean(0)) < 0.3)


def test_label_stopping_rule(orc):
    dens = W.blob_cloud(24, seed=22)
    v = orc.Volume(dens, 0.95, 0.85)
    r = v.gen_record(7, 3, rel_ci=0.05, n_min=64, n_max=200000)
    assert r["status"] == 0 and r["label"] > 0
    assert r["half_width"] <= 0.05 * r["label"]
    assert r["npaths"] >= 64
    # re-estimating with the same number of paths reproduces the label (same streams)
    rr, m, var = v.estimate_Li(7, 3, r["x"], r["d"], r["wl"], r["npaths"])
    assert abs(m - r["label"]) < 1e-12 * max(1.0, m)
    # the half-width is the normal 95 % quantile times the standard error of the mean
    from scipy import stats
    z95 = stats.norm.ppf(0.975)
    assert abs(r["half_width"] - z95 * math.sqrt(var / r["npaths"])) <= 1e-4 * r["half_width"]
    # and the rule stopped at the first path count that met it (after n_min)
    if r["npaths"] > 64:
        _, m1, var1 = v.estimate_Li(7, 3, r["x"], r["d"], r["wl"], r["npaths"] - 1)
        assert not (m1 > 0 and z95 * math.sqrt(var1 / (r["npaths"] - 1)) <= 0.05 * m1 * (1 - 1e-4))


def test_record_positions_in_a_thin_medium_follow_the_density(orc):
    """Sec. 5.1's sampler in the optically thin limit: rays with directions uniform on the
    sphere and origins uniform over the bounding sphere's cross-section are a uniform,
    isotropic flux, so first collisions fall with density proportional to mu(x) -- each
    coordinate's marginal is the trilinear ramp profile of the constant cube -- and, since the
    chords through the cube integrate to its volume from every direction, the directions of
    the rays that collide stay uniform (cos theta uniform on [-1, 1])."""
    from scipy import integrate, stats
    mu_thin = 0.01
    v = orc.Volume(np.full((N, N, N), mu_thin, np.float32), 0.5, 0.0)
    xs, dz, lz = [], [], []
    for rec in range(3000):
        r = v.gen_record(901, rec, rel_ci=1.0, n_min=1, n_max=1)
        assert r["status"] == 0
        xs.append(r["x"])
        dz.append(r["d"][2])
        lz.append(r["wl"][2])
    xs = np.array(xs)
    grid = np.linspace(0.0, 1.0, 801)
    prof = ramp(grid * N - 0.5)
    cdf = integrate.cumulative_trapezoid(prof, grid, initial=0.0)
    cdf /= cdf[-1]
    for a in range(3):
        assert stats.kstest(xs[:, a], lambda t: np.interp(t, grid, cdf)).pvalue > 1e-3, a
    assert stats.kstest(dz, stats.uniform(-1, 2).cdf).pvalue > 1e-3
    assert stats.kstest(lz, stats.uniform(-1, 2).cdf).pvalue > 1e-3
    v.close()
