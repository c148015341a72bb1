"""Pins for the oracle's quasi-distance transform (Section 2, Eq. 13-15;
Algorithm 6), each computed without the oracle's step loop:

* binary images: the largest residual of a {0, 255} image is 255 at the
  erosion that first reaches a 0 pixel, so d is the chessboard (8-conn) or
  taxicab (4-conn) distance transform of scipy.ndimage.distance_transform_cdt,
  and d is already 1-Lipschitz (eta leaves it unchanged);
* grey images: r and d from scipy's minimum filters over the clipped windows
  of every half size s (square or diamond footprint, the outside counting as
  +inf), the maximum over s and numpy's first-index argmax;
* the eta limit: the greatest 1-Lipschitz function below g, which has the
  closed form min_q g(q) + dist(p, q), by brute force over all pixel pairs;
* more erosions than qdt_steps change nothing.
"""
import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth

RNG = np.random.default_rng(1911)


def footprint(s, conn):
    if conn == 8:
        return np.ones((2 * s + 1, 2 * s + 1), bool)
    y, x = np.mgrid[-s:s + 1, -s:s + 1]
    return (np.abs(y) + np.abs(x)) <= s


def residual_reference(f, conn):
    H, W = f.shape
    S = oracle.qdt_steps(H, W, conn)
    g = f.astype(np.float64)
    if S == 0:
        return np.zeros_like(g), np.zeros(g.shape, np.int32)
    eros = [g] + [ndimage.minimum_filter(g, footprint=footprint(s, conn), mode="constant", cval=np.inf)
                  for s in range(1, S + 1)]
    res = np.stack([eros[s - 1] - eros[s] for s in range(1, S + 1)])
    r = res.max(axis=0)
    d = np.where(r > 0, res.argmax(axis=0) + 1, 0).astype(np.int32)
    return r, d


def metric(conn, dy, dx):
    return np.maximum(np.abs(dy), np.abs(dx)) if conn == 8 else np.abs(dy) + np.abs(dx)


def lipschitz_reference(g, conn):
    H, W = g.shape
    yy, xx = np.mgrid[0:H, 0:W]
    out = np.empty((H, W), np.int64)
    for y in range(H):
        for x in range(W):
            out[y, x] = (g + metric(conn, yy - y, xx - x)).min()
    return out


@pytest.mark.parametrize("conn", [4, 8])
def test_binary_qdt_is_the_distance_transform(conn):
    for H, W, p in [(1, 5, 0.5), (9, 7, 0.75), (31, 40, 0.8), (64, 64, 0.93), (6, 11, 1.0), (12, 5, 1.0)]:
        f = (RNG.random((H, W)) < p).astype(np.uint8) * 255
        if p == 1.0:
            f[0, 0] = 0  # one corner pixel: the far corner needs all qdt_steps erosions
        else:
            f[RNG.integers(H), RNG.integers(W)] = 0  # at least one background pixel
        r, d = oracle.qdt_residual(f, conn)
        dt = ndimage.distance_transform_cdt(f > 0, metric="chessboard" if conn == 8 else "taxicab")
        np.testing.assert_array_equal(d, dt)
        np.testing.assert_array_equal(r, np.where(f > 0, 255, 0))
        dl1, _ = oracle.qdt_lipschitz(d, conn)
        np.testing.assert_array_equal(dl1, d)


@pytest.mark.parametrize("conn", [4, 8])
def test_grey_residuals_match_minimum_filters(conn):
    cases = [RNG.integers(0, 256, (13, 17)).astype(np.uint8),
             synth.workload0(24, 19)["mask"],
             (RNG.integers(0, 6, (20, 22)) * 40).astype(np.uint8),  # few levels: many equal residuals
             np.full((6, 8), 77, np.uint8)]
    for f in cases:
        r, d = oracle.qdt_residual(f, conn)
        rr, dr = residual_reference(f, conn)
        np.testing.assert_array_equal(r.astype(np.float64), rr)
        np.testing.assert_array_equal(d, dr)


@pytest.mark.parametrize("conn", [4, 8])
def test_lipschitz_limit_closed_form(conn):
    for H, W, hi in [(1, 1, 5), (1, 9, 9), (8, 11, 20), (17, 13, 30)]:
        g = RNG.integers(0, hi + 1, (H, W)).astype(np.int32)
        out, _ = oracle.qdt_lipschitz(g, conn)
        np.testing.assert_array_equal(out, lipschitz_reference(g, conn))


def test_more_erosions_change_nothing():
    f = synth.workload0(21, 30)["mask"]
    for conn in (4, 8):
        S = oracle.qdt_steps(*f.shape, conn)
        r0, d0 = oracle.qdt_residual(f, conn, S)
        r1, d1 = oracle.qdt_residual(f, conn, S + 7)
        np.testing.assert_array_equal(r0, r1)
        np.testing.assert_array_equal(d0, d1)


def test_qdt_of_flat_image_is_zero():
    f = np.full((5, 6), 200, np.uint8)
    r, d, dl1 = oracle.qdt(f)
    assert not r.any() and not d.any() and not dl1.any()
