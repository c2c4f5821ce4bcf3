"""Pins for the oracle's descriptors of other stencil resolutions (the stencil-size
comparison of Sec. 7, Fig. 10): n x n x (2n - 1) points over the standard stencil's extent,
each level reading the mip matching its spacing.

- n = 5 is the standard descriptor (Sec. 4.2, Fig. 5), bit for bit in FP64 and FP32.
- Halving the spacing at the next level: level k of the n = 3 stencil and level k + 1 of
  the 5 x 5 x 9 one have the same spacing (hence the same mip) and the first's points are
  among the second's, so they read identical values; likewise the 5 x 5 x 9 stencil's level
  k inside the n = 9 stencil's level k + 1.
- A linear density is reproduced at every stencil point away from the boundary (Gaussian
  filtering and trilinear interpolation both preserve it), with the points placed at
  x + 2^(k-1) / mean * (o_x e_x + o_y e_y + o_z e_z), o = -1 + 2 i / (n - 1).
- The block input width is n^2 (2n - 1) + 1 and the network's parameter count follows."""
import math

import numpy as np
import pytest

from paper_1709_05418_gb300 import workloads as W


def unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


@pytest.fixture(scope="module")
def blob(orc):
    v = orc.Volume(W.blob_cloud(64, seed=1))
    x, d = W.random_queries((64, 64, 64), 23, seed=11, margin=0.2)
    yield v, x, d, unit([0.3, 0.5, -0.8])
    v.close()


def test_widths_and_parameter_counts(orc):
    for n in range(2, 10):
        din = orc.stencil_din(n)
        assert din == n * n * (2 * n - 1) + 1
        # per block V [200][din], W1 (blocks 2..10), b1, W2, b2; tail 200x200, 200x200, 1x200
        expect = 10 * (200 * din + 200 + 200 * 200 + 200) + 9 * 200 * 200 + 2 * (200 * 200 + 200) + 201
        assert orc.net_param_count(din=din) == expect == W.param_count(din=din)
    assert orc.stencil_din(5) == orc.DIN and orc.net_param_count(din=orc.DIN) == 1296601
    for n in (1, 10):
        with pytest.raises(ValueError):
            orc.stencil_din(n)


def test_five_is_the_standard_stencil(blob):
    v, x, d, wl = blob
    assert np.array_equal(v.descriptor_stencil(5, x, d, wl), v.descriptor(x, d, wl))
    x32, d32, wl32 = x.astype(np.float32), d.astype(np.float32), wl.astype(np.float32)
    assert np.array_equal(v.descriptor_stencil(5, x32, d32, wl32, f32=True),
                          v.descriptor(x32, d32, wl32, f32=True))


def _index(n, ix, iy, iz):
    return (iz * n + iy) * n + ix


@pytest.mark.parametrize("f32", [False, True])
def test_halved_spacing_at_the_next_level_reads_the_same_points(blob, f32):
    v, x, d, wl = blob
    if f32:
        x, d, wl = x.astype(np.float32), d.astype(np.float32), wl.astype(np.float32)
    z3 = v.descriptor_stencil(3, x, d, wl, f32=f32)
    z5 = v.descriptor_stencil(5, x, d, wl, f32=f32)
    z9 = v.descriptor_stencil(9, x, d, wl, f32=f32)
    nonzero = 0
    for k in range(9):                               # 0-based level k and k + 1
        for iz in range(5):
            for iy in range(3):
                for ix in range(3):
                    # n = 3 offset -1 + i is twice the n = 5 offset at the next level: -1 + (i + 1)/2
                    a = z3[:, k, _index(3, ix, iy, iz)]
                    b = z5[:, k + 1, _index(5, ix + 1, iy + 1, iz + 1)]
                    assert np.array_equal(a, b), (k, ix, iy, iz)
                    nonzero += int(np.count_nonzero(a))
        for iz in range(9):
            for iy in range(5):
                for ix in range(5):
                    # n = 5 offset -1 + i/2 is twice the n = 9 offset -1 + (i + 2)/4
                    a = z5[:, k, _index(5, ix, iy, iz)]
                    b = z9[:, k + 1, _index(9, ix + 2, iy + 2, iz + 2)]
                    assert np.array_equal(a, b), (k, ix, iy, iz)
    assert nonzero > 1000
    # gamma closes every level's block
    assert np.array_equal(z3[:, :, -1], z5[:, :, -1]) and np.array_equal(z5[:, :, -1], z9[:, :, -1])


@pytest.mark.parametrize("n", [2, 3, 4, 7])
def test_linear_density_is_reproduced(orc, n):
    g = 96
    i = np.arange(g, dtype=np.float64)
    Z, Y, X = np.meshgrid(i, i, i, indexing="ij")
    a, b, c, e = 30.0, 0.25, -0.125, 0.0625     # exact in FP32
    v = orc.Volume((a + b * X + c * Y + e * Z).astype(np.float32))
    st = v.stats()
    mean, inv_mean = st["mean"], st["inv_mean"]
    h = 2.0 / (n - 1)
    rng = np.random.default_rng(4)
    checked = 0
    for _ in range(4):
        x = rng.uniform(0.4, 0.6, size=3)
        dd = unit(rng.normal(size=3))
        wl = unit(rng.normal(size=3))
        z = v.descriptor_stencil(n, x[None], dd[None], wl)[0]
        ez = wl
        ex = unit(np.cross(ez, -dd))
        ey = np.cross(ez, ex)
        for k in range(1, 11):
            # mip: the largest power of two (fine voxels) not above the spacing h 2^(k-1) mfp
            sk = h * 2.0 ** (k - 1) * st["inv_mean_f"] * g
            m = min(max(math.floor(math.log2(sk)), 0), st["levels"] - 1)
            reach = 3 * 2 ** m + 2 ** m + 1
            for iz in range(2 * n - 1):
                for iy in range(n):
                    for ix in range(n):
                        o = np.array([-1 + h * ix, -1 + h * iy, -1 + h * iz])
                        p = x + 2 ** (k - 1) * inv_mean * (o[0] * ex + o[1] * ey + o[2] * ez)
                        u = p * g - 0.5
                        if np.all(u > reach) and np.all(u < g - 1 - reach):
                            exp = (a + b * u[0] + c * u[1] + e * u[2]) / mean
                            got = z[k - 1, _index(n, ix, iy, iz)]
                            assert abs(got - exp) <= 1e-11 * abs(exp), (n, k, ix, iy, iz, got, exp)
                            checked += 1
            assert abs(z[k - 1, -1] - math.acos(np.clip(np.dot(-dd, wl), -1, 1))) < 1e-12
    assert checked > 20 * n


def test_f32_matches_f64(blob):
    v, x, d, wl = blob
    for n in (3, 7):
        z64 = v.descriptor_stencil(n, x, d, wl)
        z32 = v.descriptor_stencil(n, x.astype(np.float32), d.astype(np.float32), wl.astype(np.float32), f32=True)
        assert np.abs(z32.astype(np.float64) - z64).max() < 2e-5 * max(1.0, np.abs(z64).max())
