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


def test_lorenz_mie_single_scattering_matches_quadrature(orc):
    """With the table as the phase function, a front-lit slab pixel's single scattering
    follows the same 1-D quadrature as with HG (the phase value enters as p(cos theta))."""
    from paper_1709_05418_gb300 import workloads as W
    n = 8
    vol = orc.Volume(np.full((n, n, n), 1.5, np.float32), 0.9, 0.85)
    vol.set_phase_lm(True)
    cam = W.camera((n, n, n), 4, 4, spp=1, seed=3, light_seed=4)
    a = vol.render_pixels(cam, np.arange(16), params=None)
    vol.set_phase_lm(False)
    b = vol.render_pixels(cam, np.arange(16), params=None)
    assert np.isfinite(a).all() and not np.allclose(a, b)
    vol.close()
