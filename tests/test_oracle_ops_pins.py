"""Pins for the oracle's geodesic operators (Section 2, Eq. 6-12).

On binary images each operator reduces to a textbook set operation that
scipy computes independently of the oracle's step loop:
  HFILL    -> scipy.ndimage.binary_fill_holes (holes = background components
              that do not reach the border, under the connectivity used);
  RAOBJ    -> remove the foreground components (label) that touch the border;
  gamma_rec^s -> keep the foreground components that meet the erosion of the
              image by the (2s+1)^2 square (binary_erosion, outside = 1).
On grey images: HMAX against the widest-path reconstruction of f - h under
f, DOME = f - HMAX, and a constructed image whose peak heights are known.
"""
import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth
from tests.test_oracle_pins import widest_path_reconstruct

RNG = np.random.default_rng(2718)


def structure(conn):
    return ndimage.generate_binary_structure(2, 2 if conn == 8 else 1)


def random_binary(H, W, p=0.45):
    return (RNG.random((H, W)) < p).astype(np.uint8) * 255


@pytest.mark.parametrize("conn", [4, 8])
def test_hfill_binary_is_fill_holes(conn):
    for H, W in [(1, 1), (5, 7), (30, 41), (64, 64)]:
        f = random_binary(H, W)
        ref = ndimage.binary_fill_holes(f > 0, structure=structure(conn)).astype(np.uint8) * 255
        np.testing.assert_array_equal(oracle.hfill(f, conn=conn), ref)


@pytest.mark.parametrize("conn", [4, 8])
def test_raobj_binary_removes_border_components(conn):
    for H, W in [(1, 1), (6, 5), (33, 47), (64, 64)]:
        f = random_binary(H, W, 0.5)
        lab, _ = ndimage.label(f > 0, structure=structure(conn))
        border = np.unique(np.concatenate([lab[0], lab[-1], lab[:, 0], lab[:, -1]]))
        border = border[border > 0]
        ref = np.where(np.isin(lab, border), 0, f).astype(np.uint8)
        np.testing.assert_array_equal(oracle.raobj(f, conn=conn), ref)


@pytest.mark.parametrize("conn", [4, 8])
def test_open_rec_binary_keeps_components_meeting_the_erosion(conn):
    for H, W in [(7, 9), (40, 37), (64, 80)]:
        f = random_binary(H, W, 0.6)
        for s in (1, 2, 3):
            ero = ndimage.binary_erosion(f > 0, structure=np.ones((2 * s + 1, 2 * s + 1), bool), border_value=1)
            lab, _ = ndimage.label(f > 0, structure=structure(conn))
            keep = np.unique(lab[ero])
            keep = keep[keep > 0]
            ref = np.where(np.isin(lab, keep), f, 0).astype(np.uint8)
            np.testing.assert_array_equal(oracle.open_rec(f, s, conn=conn), ref)


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("kind", ["u8", "f64"])
def test_hmax_is_widest_path_of_shifted_marker(conn, kind):
    for H, W in [(12, 9), (25, 31)]:
        if kind == "u8":
            f = RNG.integers(0, 256, (H, W)).astype(np.uint8)
            h = 37
            mk = np.maximum(f.astype(np.float64) - h, 0)
        else:
            f = RNG.random((H, W))
            h = 0.21
            mk = f - h
        ref = widest_path_reconstruct(mk, f.astype(np.float64), conn, "dilate")
        got = oracle.hmax(f, h, conn=conn)
        np.testing.assert_array_equal(got.astype(np.float64), ref)
        np.testing.assert_array_equal(oracle.dome(f, h, conn=conn).astype(np.float64),
                                      f.astype(np.float64) - ref)


def test_hmax_flattens_peaks_lower_than_h():
    """Background 10 with square plateaus of heights 30, 60, 100 (known
    regional maxima): HMAX_h lowers each plateau by h or to the background."""
    f = np.full((40, 60), 10, np.uint8)
    f[5:10, 5:10] = 30
    f[20:26, 20:26] = 60
    f[30:35, 45:52] = 100
    out = oracle.hmax(f, 40)
    assert np.all(out[f == 10] == 10)
    assert np.all(out[5:10, 5:10] == 10)      # 20 above the background < 40: removed
    assert np.all(out[20:26, 20:26] == 20)    # 60 - 40
    assert np.all(out[30:35, 45:52] == 60)    # 100 - 40
    dome = oracle.dome(f, 40)
    assert dome.max() == 40 and dome[5:10, 5:10].max() == 20


def test_operators_on_workload_image_invariants():
    g = synth.workload0(96, 80)["mask"]
    fill = oracle.hfill(g)
    assert np.all(fill >= g)
    np.testing.assert_array_equal(fill[0], g[0])
    np.testing.assert_array_equal(oracle.hfill(fill), fill)  # idempotent
    ra = oracle.raobj(g)
    assert np.all(ra <= g)
    op = oracle.open_rec(g, 3)
    assert np.all(op <= g)
    np.testing.assert_array_equal(oracle.open_rec(op, 3), op)  # idempotent


def test_hmax_of_image_lower_than_h():
    """An image whose values all lie below h: the marker f - h is below the
    image everywhere; uint8 saturates it at 0, floats keep f - h, and the
    reconstruction under f then returns that marker's maximum reachable value."""
    f = np.full((9, 11), 10, np.uint8)
    f[4, 5] = 25
    np.testing.assert_array_equal(oracle.hmax(f, 40), np.zeros_like(f))
    np.testing.assert_array_equal(oracle.dome(f, 40), f)
    g = f.astype(np.float64)
    np.testing.assert_array_equal(oracle.hmax(g, 40.0), np.full_like(g, -15.0))
