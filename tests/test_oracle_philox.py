"""Pins of the oracle's Philox4x32-10 and uniform conversion (CPU)."""
import os

import numpy as np

from oracle import oracle as orc

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    n = 0
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        out = orc.philox4x32_10(w[0:4], w[4:6])
        assert [int(x) for x in out] == w[6:10], line
        n += 1
    assert n == 3


def test_u53_exact_endpoints():
    assert orc.u53(0, 0) == 0.0
    assert orc.u53(0x80000000, 0) == 0.5
    assert orc.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    # the low 11 bits of the second word are dropped
    assert orc.u53(0, 0x7FF) == 0.0
    assert orc.u53(0, 0x800) == 2.0 ** -53


def test_philox_counter_sensitivity_and_uniformity():
    # every output byte of 20000 consecutive counters: chi^2 over 256 bins
    out = np.array([orc.philox4x32_10([i, 7, 0, 1 << 24], [42, 0]) for i in range(20000)],
                   dtype=np.uint32)
    b = out.view(np.uint8).ravel()
    h = np.bincount(b, minlength=256)
    e = b.size / 256.0
    chi2 = ((h - e) ** 2 / e).sum()
    assert 170 < chi2 < 350, chi2          # 255 dof, ~5 sigma band
    # flipping one counter bit changes ~half the output bits
    a = orc.philox4x32_10([1, 2, 3, 4], [5, 6])
    c = orc.philox4x32_10([1, 2, 3, 5], [5, 6])
    flips = sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, c))
    assert 40 < flips < 90
