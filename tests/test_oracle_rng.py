"""Pins for the oracle's counter-based generator (Philox4x32-10, Salmon et al. 2011)."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox_known_answers(orc):
    n = 0
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        assert orc.philox4x32_10(w[:4], w[4:6]) == w[6:]
        n += 1
    assert n == 3


def test_philox_uniformity(orc):
    # 4096 blocks -> 16384 words: top-24-bit uniforms pass a coarse chi-square
    vals = []
    for i in range(4096):
        vals += orc.philox4x32_10([i, 7, 0, 2], [12345, 0])
    u = (np.array(vals) >> 8) * 2.0 ** -24
    assert u.min() >= 0.0 and u.max() < 1.0
    hist, _ = np.histogram(u, bins=32, range=(0, 1))
    e = u.size / 32
    chi2 = ((hist - e) ** 2 / e).sum()
    assert chi2 < 70.0  # 31 dof, p ~ 1e-4
