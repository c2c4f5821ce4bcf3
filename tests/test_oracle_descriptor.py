"""Pins for the oracle's hierarchical stencil descriptor (Sec. 4.2, Fig. 5)."""
import math

import numpy as np

from paper_1709_05418_gb300 import workloads as W


def unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def test_frame_geometry(orc):
    rng = np.random.default_rng(3)
    for _ in range(200):
        d = unit(rng.normal(size=3))
        wl = unit(rng.normal(size=3))
        ex, ey, ez, gam = orc.frame(d, wl)
        w = -d                                   # propagation direction (Eq. 1)
        M = np.stack([ex, ey, ez])
        assert np.allclose(M @ M.T, np.eye(3), atol=1e-12)
        assert np.allclose(ez, wl, atol=0)       # z towards the light
        assert abs(np.dot(ex, w)) < 1e-12        # x normal to the plane of z and omega
        assert np.allclose(np.cross(ex, ey), ez, atol=1e-12)   # right-handed
        assert abs(gam - math.acos(np.clip(np.dot(w, wl), -1, 1))) < 1e-12
        # omega lies in the (y, z) plane with a negative y component
        assert abs(np.dot(w, ey) + math.sin(gam)) < 1e-12
    # degenerate: omega parallel to the light
    ex, ey, ez, gam = orc.frame(np.array([0, 0, -1.0]), np.array([0, 0, 1.0]))
    M = np.stack([ex, ey, ez])
    assert np.allclose(M @ M.T, np.eye(3), atol=1e-12) and gam == 0.0


def _stencil_world(x, d, wl, inv_mean, k):
    """World positions of the 225 points of level k (1-based), (iz*5+iy)*5+ix order."""
    w = -unit(d)
    ez = unit(wl)
    ex = unit(np.cross(ez, w))
    ey = np.cross(ez, ex)
    pts = []
    for iz in range(9):
        for iy in range(5):
            for ix in range(5):
                o = np.array([-1 + 0.5 * ix, -1 + 0.5 * iy, -1 + 0.5 * iz])
                pts.append(x + 2 ** (k - 1) * inv_mean * (o[0] * ex + o[1] * ey + o[2] * ez))
    return np.array(pts)


def test_constant_volume(orc):
    n = 64
    v = orc.Volume(np.full((n, n, n), 40.0, np.float32))   # mfp = 1/40 = 2.56 voxels
    st = v.stats()
    assert st["mean"] == 40.0
    x = np.array([[0.5, 0.5, 0.5]])
    d = np.array([[0.3, -0.2, 0.9]])
    wl = unit([0.1, 0.8, -0.3])
    z = v.descriptor(x, unit(d[0])[None], wl)[0]
    z32 = v.descriptor(x, unit(d[0])[None], wl, f32=True)[0]
    for k in range(1, 11):
        pts = _stencil_world(x[0], d[0], wl, 1 / 40.0, k)
        m = st["mip_of_level"][k - 1]
        h = 2 ** m / n
        # support of Gaussian + trilinear neighbourhood, in world units
        reach = (3 * 2 ** m + 2 ** m + 1) / n
        inside = np.all((pts > reach) & (pts < 1 - reach), axis=1)
        outside = np.any((pts < -2 * h - 3 * 2 ** m / n) | (pts > 1 + 2 * h + 3 * 2 ** m / n), axis=1)
        vals = z[k - 1, :225]
        assert np.all(np.abs(vals[inside] - 1.0) < 1e-12)
        assert np.all(np.abs(z32[k - 1, :225][inside] - 1.0) < 2e-6)
        assert np.all(vals[outside] == 0.0) and np.all(z32[k - 1, :225][outside] == 0.0)
        if k <= 2:
            assert inside.all()
        if k >= 8:
            assert outside.any()
        assert z[k - 1, 225] == z[0, 225]


def test_linear_density_is_reproduced(orc):
    # Gaussian filtering and trilinear interpolation both reproduce a linear field, so
    # away from the boundary every stencil entry equals the field at the stencil point
    n = 96
    i = np.arange(n, dtype=np.float64)
    Z, Y, X = np.meshgrid(i, i, i, indexing="ij")
    a, b, c, e = 30.0, 0.25, -0.125, 0.0625     # exact in FP32
    dens = (a + b * X + c * Y + e * Z).astype(np.float32)
    v = orc.Volume(dens)
    st = v.stats()
    mean = st["mean"]
    rng = np.random.default_rng(4)
    checked = 0
    for _ in range(6):
        x = rng.uniform(0.4, 0.6, size=3)
        d = unit(rng.normal(size=3))
        wl = unit(rng.normal(size=3))
        z = v.descriptor(x[None], d[None], wl)[0]
        for k in range(1, 11):
            m = st["mip_of_level"][k - 1]
            pts = _stencil_world(x, d, wl, st["inv_mean"], k)
            u = pts * n - 0.5                           # fine voxel coordinates
            reach = 3 * 2 ** m + 2 ** m + 1
            ok = np.all((u > reach) & (u < n - 1 - reach), axis=1)
            exp = (a + b * u[:, 0] + c * u[:, 1] + e * u[:, 2]) / mean
            assert np.allclose(z[k - 1, :225][ok], exp[ok], rtol=1e-11, atol=0)
            checked += int(ok.sum())
        assert abs(z[0, 225] - math.acos(np.clip(np.dot(-d, wl), -1, 1))) < 1e-12
    assert checked > 2000


def test_f32_matches_f64(orc):
    dens = W.blob_cloud(32, seed=11)
    v = orc.Volume(dens)
    x, d = W.random_queries(dens.shape, 64, seed=12)
    wl = unit([0.3, 0.5, -0.8])
    z64 = v.descriptor(x, d, wl)
    z32 = v.descriptor(x.astype(np.float32), d.astype(np.float32), wl.astype(np.float32), f32=True)
    err = np.abs(z32.astype(np.float64) - z64)
    scale = max(1.0, np.abs(z64).max())
    assert err.max() < 2e-5 * scale


def test_rotation_invariance(orc):
    # a cyclic permutation of the axes is a rotation: rotating the grid, the query and
    # the light together leaves the descriptor unchanged
    dens = W.blob_cloud(32, seed=13)
    # rot[z', y', x'] = dens[y', x', z']: a point (x, y, z) moves to (y, z, x)
    rot = np.ascontiguousarray(np.transpose(dens, (2, 0, 1)))
    v0, v1 = orc.Volume(dens), orc.Volume(rot)
    x, d = W.random_queries(dens.shape, 16, seed=14)
    wl = unit([0.2, -0.7, 0.4])
    P = lambda a: np.asarray(a)[..., [1, 2, 0]]
    z0 = v0.descriptor(x, d, wl)
    z1 = v1.descriptor(P(x), P(d), P(wl))
    assert np.allclose(z0, z1, rtol=1e-10, atol=1e-12)


def test_level_extent_ratio(orc):
    # level 10 spans 2^9 times the extent of level 1 (volume ratio (2^9)^3 ~ 1.3e8)
    pts1 = _stencil_world(np.zeros(3), unit([1, 2, 3]), unit([0, 0, 1]), 1.0, 1)
    pts10 = _stencil_world(np.zeros(3), unit([1, 2, 3]), unit([0, 0, 1]), 1.0, 10)
    e1 = np.ptp(pts1 @ np.eye(3), axis=0)
    e10 = np.ptp(pts10 @ np.eye(3), axis=0)
    assert np.allclose(e10, 512 * e1)
    assert abs(np.prod(e10) / np.prod(e1) - 512 ** 3) < 1e-3 * 512 ** 3


def test_blended_mips_reproduce_a_linear_field(orc):
    """With blending on, each entry is (1 - w) rho_m + w rho_{m+1} read at the same world
    point; both levels of a linear field are that field away from the boundary, so the
    blend reproduces it too -- a wrong level, scale or coordinate for level m + 1 would not."""
    n = 96
    i = np.arange(n, dtype=np.float64)
    Z, Y, X = np.meshgrid(i, i, i, indexing="ij")
    a, b, c, e = 30.0, 0.25, -0.125, 0.0625
    dens = (a + b * X + c * Y + e * Z).astype(np.float32)
    v = orc.Volume(dens)
    v.set_mip_blend(True)
    st = v.stats()
    assert any(0.05 < w < 0.95 for w in st["mip_weight"])
    rng = np.random.default_rng(4)
    checked = 0
    for _ in range(6):
        x = rng.uniform(0.4, 0.6, size=3)
        d = unit(rng.normal(size=3))
        wl = unit(rng.normal(size=3))
        z = v.descriptor(x[None], d[None], wl)[0]
        for k in range(1, 11):
            m = st["mip_of_level"][k - 1] + 1
            pts = _stencil_world(x, d, wl, st["inv_mean"], k)
            u = pts * n - 0.5
            reach = 3 * 2 ** m + 2 ** m + 1
            ok = np.all((u > reach) & (u < n - 1 - reach), axis=1)
            exp = (a + b * u[:, 0] + c * u[:, 1] + e * u[:, 2]) / st["mean"]
            assert np.allclose(z[k - 1, :225][ok], exp[ok], rtol=1e-11, atol=0)
            checked += int(ok.sum())
    assert checked > 500


def test_blended_mips_are_continuous_across_a_level_switch(orc):
    """Scaling the extinction by c moves the stencil spacing (in voxels) as 1/c; where it
    crosses a power of two the selected level switches.  Without blending the descriptor
    jumps there, with blending it moves by O(dc)."""
    base = W.blob_cloud(48, nblobs=6, seed=21)
    v0 = orc.Volume(base)
    st = v0.stats()
    k = 2                                         # stencil level 3 (0-based 2)
    sk = 0.5 * math.ldexp(st["inv_mean_f"], k) * st["inv_h0"]
    j = math.floor(math.log2(sk))
    c_switch = sk / 2.0 ** j                      # spacing / c crosses 2^j at c = c_switch
    x, d = W.random_queries(base.shape, 16, seed=3, margin=0.25)
    wl = unit([0.2, 0.9, -0.3])
    out = {}
    for blend in (False, True):
        zs = []
        for f in (1.0 - 1e-4, 1.0 + 1e-4):
            v = orc.Volume(base * np.float32(c_switch * f))
            v.set_mip_blend(blend)
            zs.append(v.descriptor(x, d, wl)[:, k, :225])
            assert v.stats()["mip_of_level"][k] == (j - 1 if f > 1 else j) or not (0 < j < st["levels"])
            v.close()
        out[blend] = np.abs(zs[1] - zs[0]).max() / np.abs(zs[0]).max()
    assert out[False] > 1e-2, out
    assert out[True] < 2e-3, out
