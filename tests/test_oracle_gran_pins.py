"""Pins for the oracle's openings, closings, granulometry, pattern spectrum and
alternating sequential filters (Section 2, Eq. 16-20), computed without the
oracle's step loop:

* gamma_s / phi_s against scipy's minimum and maximum filters over the
  (2s+1)^2 square, composed in the order of Eq. 16 / 19, with the outside of
  the image counting as +inf for the minimum and -inf for the maximum (the
  clipped window);
* ASF_s against the same scipy compositions in the order of Eq. 20;
* G_s of a binary image of separated squares: a square of side a survives
  gamma_s exactly when a >= 2s + 1, so G_s = 255 * sum of a^2 over those.
"""
import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth

RNG = np.random.default_rng(16)


def sc_erode(g, s):
    return ndimage.minimum_filter(g, size=2 * s + 1, mode="constant", cval=np.inf) if s else g


def sc_dilate(g, s):
    return ndimage.maximum_filter(g, size=2 * s + 1, mode="constant", cval=-np.inf) if s else g


def sc_open(g, s):
    return sc_dilate(sc_erode(g, s), s)


def sc_close(g, s):
    return sc_erode(sc_dilate(g, s), s)


def grey_cases():
    return [RNG.integers(0, 256, (1, 23)).astype(np.uint8), RNG.integers(0, 256, (17, 1)).astype(np.uint8),
            synth.workload0(29, 35)["mask"], RNG.integers(0, 256, (24, 19)).astype(np.uint8),
            RNG.random((13, 21)).astype(np.float32)]


def test_opening_and_closing_match_scipy():
    for f in grey_cases():
        g = f.astype(np.float64)
        for s in range(0, 5):
            np.testing.assert_array_equal(oracle.opening(f, s).astype(np.float64), sc_open(g, s))
            np.testing.assert_array_equal(oracle.closing(f, s).astype(np.float64), sc_close(g, s))


def test_asf_matches_scipy_composition():
    for f in grey_cases():
        for s in range(0, 4):
            g = f.astype(np.float64)
            for k in range(1, s + 1):
                g = sc_close(sc_open(g, k), k)
            np.testing.assert_array_equal(oracle.asf(f, s).astype(np.float64), g)


def test_granulometry_matches_scipy_sums():
    for f in grey_cases()[:4]:
        G, PS = oracle.granulometry(f, 5)
        ref = np.array([sc_open(f.astype(np.float64), s).sum() for s in range(6)])
        np.testing.assert_array_equal(G, ref)
        np.testing.assert_array_equal(PS, ref[:-1] - ref[1:])


def test_granulometry_of_separated_squares():
    f = np.zeros((60, 80), np.uint8)
    sides = []
    y = 1
    for row in ([3, 5, 8, 11], [1, 2, 7, 9, 4]):
        x = 1
        for a in row:
            f[y:y + a, x:x + a] = 255
            sides.append(a)
            x += a + 2
        y += max(row) + 2
    G, PS = oracle.granulometry(f, 6)
    for s in range(7):
        assert G[s] == 255 * sum(a * a for a in sides if a >= 2 * s + 1), s
    assert np.all(PS >= 0)
