"""Pins for the oracle's volume statistics (Sec. 4.2 mean over non-zero voxels) and
its Gaussian mip pyramid (Sec. 6, sigma_i = 2^i fine voxels)."""
import math

import numpy as np
import pytest


def vol(orc, d, albedo=0.99, g=0.85):
    return orc.Volume(np.asarray(d, np.float32), albedo, g)


def test_stats_exact_on_hand_grid(orc):
    d = np.zeros((4, 4, 4), np.float32)
    d[0, 0, 0], d[1, 2, 3], d[3, 3, 3], d[2, 1, 0] = 1.0, 2.0, 3.5, 0.25
    st = vol(orc, d).stats()
    assert st["nonzero"] == 4
    assert st["majorant"] == 3.5
    assert st["mean"] == 6.75 / 4          # dyadic values: fixed point is exact
    assert st["inv_mean_f"] == np.float32(4 / 6.75)
    assert st["levels"] == 3               # 4 -> 2 -> 1
    assert st["h0"] == 0.25 and st["ext"] == (1.0, 1.0, 1.0)


def test_stats_mean_close_to_extended_sum(orc):
    rng = np.random.default_rng(0)
    d = rng.uniform(0, 50, size=(20, 17, 23)).astype(np.float32)
    d[d < 20] = 0
    st = vol(orc, d).stats()
    ref = d[d > 0].astype(np.float64).mean()
    assert abs(st["mean"] - ref) <= 1e-8 * ref
    assert abs(st["mean_ld"] - ref) <= 1e-12 * ref
    assert st["nonzero"] == int((d > 0).sum())
    # non-cubic: longest edge spans the unit box
    assert st["inv_h0"] == 23 and st["ext"] == (1.0, 17 / 23, 20 / 23)


def test_level_count_and_dims(orc):
    for n, L in [(1, 1), (2, 2), (64, 7), (65, 8), (160, 9)]:
        d = np.ones((1, 1, n), np.float32)
        st = vol(orc, d).stats()
        assert st["levels"] == L, (n, st["levels"])
        assert st["dims"][L - 1][0] == 1
        assert st["dims"][1][0] == (n + 1) // 2 if L > 1 else True


def test_mip_level_choice_brackets_stencil_spacing(orc):
    # stencil spacing at level k is 0.5 * 2^(k-1) mean free paths; the chosen mip
    # level's voxel is the largest power of two (in fine voxels) not above it
    rng = np.random.default_rng(1)
    for peak in (0.5, 5.0, 50.0, 500.0):
        d = (rng.uniform(0, 1, (32, 32, 32)) * peak).astype(np.float32)
        st = vol(orc, d).stats()
        L = st["levels"]
        for k in range(10):
            s = 0.5 * 2 ** k * float(st["inv_mean_f"]) * st["inv_h0"]
            m = st["mip_of_level"][k]
            if 0 < m < L - 1:
                assert 2 ** m <= s < 2 ** (m + 1)
            elif m == 0:
                assert s < 2
            else:
                assert s >= 2 ** (L - 1)
        assert st["mip_of_level"] == sorted(st["mip_of_level"])


def test_gauss_taps(orc):
    for lv in range(6):
        w, off = orc.gauss_taps(lv)
        T = 7 if lv == 0 else 6 * 2 ** lv
        assert w.size == T
        assert abs(w.sum() - 1.0) < 1e-14
        assert np.allclose(w, w[::-1], rtol=0, atol=1e-17)
        assert np.argmax(w) in (T // 2 - 1, T // 2)
        # tap t of output j is fine voxel j*2^lv + off + m, centred on (j+0.5)2^lv - 0.5
        centre = 0 if lv == 0 else 2 ** lv / 2 - 0.5
        offs = off + np.arange(T) - centre
        assert abs(np.dot(w, offs)) < 1e-12
        assert offs.max() <= 3 * 2 ** lv + 1e-12 and offs.min() >= -3 * 2 ** lv - 1e-12


def test_constant_volume_interior_is_one(orc):
    n = 40
    v = vol(orc, np.full((n, n, n), 7.25, np.float32))
    for lv in (0, 1, 2):
        m64 = v.mip_level(lv)
        m32 = v.mip_level(lv, f32=True)
        step, r = 2 ** lv, 3 * 2 ** lv
        for j in range(m64.shape[0]):
            c = (j + 0.5) * step - 0.5
            if c - r >= 0 and c + r <= n - 1:
                assert abs(m64[j, j, j] - 1.0) < 1e-12
                assert abs(m32[j, j, j] - 1.0) < 1e-5
        # zero padding outside the grid: the corner loses mass
        assert m64[0, 0, 0] < 1.0


def _brute_level(d, lv):
    """3-D direct (non-separable) sum of the truncated, normalised Gaussian."""
    sig = 2.0 ** lv
    nz, ny, nx = d.shape
    dims = [(s + 2 ** lv - 1) // 2 ** lv for s in (nz, ny, nx)]
    out = np.zeros(dims)
    for jz in range(dims[0]):
        for jy in range(dims[1]):
            for jx in range(dims[2]):
                cs = [(j + 0.5) * 2 ** lv - 0.5 if lv else float(j) for j in (jz, jy, jx)]
                ws = []
                for c, nn in zip(cs, (nz, ny, nx)):
                    t = np.arange(math.floor(c - 3 * sig), math.ceil(c + 3 * sig) + 1)
                    t = t[np.abs(t - c) <= 3 * sig + 1e-9]
                    w = np.exp(-(t - c) ** 2 / (2 * sig * sig))
                    w /= w.sum()
                    keep = (t >= 0) & (t < nn)
                    ws.append((t[keep], w[keep]))
                (tz, wz), (ty, wy), (tx, wx) = ws
                blk = d[np.ix_(tz, ty, tx)].astype(np.float64)
                out[jz, jy, jx] = np.einsum("zyx,z,y,x->", blk, wz, wy, wx)
    return out


def test_separable_matches_brute_force(orc):
    rng = np.random.default_rng(2)
    d = rng.uniform(0, 3, size=(8, 9, 10)).astype(np.float32)
    v = vol(orc, d)
    mean = v.stats()["mean"]
    for lv in (0, 1, 2):
        ref = _brute_level(d, lv) / mean
        got = v.mip_level(lv)
        assert got.shape == ref.shape
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14)
        got32 = v.mip_level(lv, f32=True)
        np.testing.assert_allclose(got32, ref, rtol=2e-6, atol=1e-7)


def test_linear_field_preserved_in_interior(orc):
    n = 48
    i = np.arange(n, dtype=np.float64)
    Z, Y, X = np.meshgrid(i, i, i, indexing="ij")
    d = (10.0 + 0.25 * X - 0.125 * Y + 0.0625 * Z).astype(np.float32)
    v = vol(orc, d)
    mean = v.stats()["mean"]
    for lv in (1, 2):
        m = v.mip_level(lv)
        step, r = 2 ** lv, 3 * 2 ** lv
        for j in range(m.shape[0]):
            c = (j + 0.5) * step - 0.5
            if c - r >= 0 and c + r <= n - 1:
                exp = (10.0 + 0.25 * c - 0.125 * c + 0.0625 * c) / mean
                assert abs(m[j, j, j] - exp) < 1e-12 * exp


def test_gaussian_blob_variances_add(orc):
    # a sampled Gaussian of width s filtered by sigma = 2^lv is (to the truncation of
    # the kernel at 3 sigma) a Gaussian of variance s^2 + sigma^2
    n, s, lv = 48, 3.0, 1
    c0 = 22.5                                   # level-1 cell j = 11: (11 + 0.5) * 2 - 0.5
    i = np.arange(n, dtype=np.float64)
    Z, Y, X = np.meshgrid(i, i, i, indexing="ij")
    d = np.exp(-((X - c0) ** 2 + (Y - c0) ** 2 + (Z - c0) ** 2) / (2 * s * s)).astype(np.float32)
    v = vol(orc, d)
    mean = v.stats()["mean"]
    m = v.mip_level(lv) * mean
    sig2 = s * s + 4.0
    assert abs(m[11, 11, 11] - (s * s / sig2) ** 1.5) < 0.02 * (s * s / sig2) ** 1.5
    # second moment along x of the decimated result
    cx = (np.arange(m.shape[2]) + 0.5) * 2 - 0.5 - c0
    prof = m[11, 11, :]
    var = (prof * cx ** 2).sum() / prof.sum()
    assert abs(var - sig2) < 0.02 * sig2


def test_rejects_bad_volumes(orc):
    with pytest.raises(ValueError):
        vol(orc, np.zeros((4, 4, 4)))
    bad = np.ones((4, 4, 4), np.float32)
    bad[1, 1, 1] = -1
    with pytest.raises(ValueError):
        vol(orc, bad)
    bad[1, 1, 1] = np.nan
    with pytest.raises(ValueError):
        vol(orc, bad)
