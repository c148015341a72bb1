"""GPU quasi-distance transform (Section 2, Eq. 13-15; Algorithm 6) against
the oracle, through the C ABI entry point geo_qdt.

* Sizes the oracle finishes in seconds, spanning several register tiles and a
  ragged tail, conn 4 and 8: r, d and d_l1 element by element.
* 1024x1024 (the workload-1 image and a binary image): properties that fix
  the result at any size -- on the binary image d is scipy's chessboard
  distance transform; on the grey image r and d of sampled pixels follow from
  the minima of f over the rings around them, and d_l1 at sampled pixels is
  min_q d(q) + dist(p, q), with d_l1 <= d and 1-Lipschitz everywhere.
"""
import ctypes

import numpy as np
import pytest
import torch
from scipy import ndimage

import oracle
import synth

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(13074)


def gm():
    import paper_1911_13074_gb300 as m
    return m


def run(f, conn):
    r, d, dl1 = gm().qdt(torch.from_numpy(f).cuda(), conn=conn)
    torch.cuda.synchronize()
    assert gm().device_status() == 0
    return r.cpu().numpy(), d.cpu().numpy(), dl1.cpu().numpy()


def images(H, W):
    return {"workload": synth.workload0(H, W)["mask"],
            "noise": RNG.integers(0, 256, (H, W)).astype(np.uint8),
            "levels": (RNG.integers(0, 5, (H, W)) * 50).astype(np.uint8),
            "binary": (RNG.random((H, W)) < 0.97).astype(np.uint8) * 255}


@pytest.mark.parametrize("conn", [8, 4])
@pytest.mark.parametrize("H,W", [(1, 1), (1, 37), (29, 1), (5, 7), (97, 131), (260, 301)])
def test_qdt_matches_oracle(H, W, conn):
    for name, f in images(H, W).items():
        if conn == 4 and H * W > 20000 and name != "workload":
            continue  # the oracle's H + W - 2 erosions: keep the CPU time bounded
        r, d, dl1 = run(f, conn)
        ro, do_, dlo = oracle.qdt(f, conn)
        np.testing.assert_array_equal(r, ro, err_msg=f"r {name}")
        np.testing.assert_array_equal(d, do_, err_msg=f"d {name}")
        np.testing.assert_array_equal(dl1, dlo, err_msg=f"d_l1 {name}")


def ring_profile(f, y, x):
    """eps_s(f)(p) for s = 0..max(H, W) - 1 from the minima of f over the
    rings max(|dy|, |dx|) = s around p (the clipped square windows)."""
    H, W = f.shape
    yy, xx = np.mgrid[0:H, 0:W]
    k = np.maximum(np.abs(yy - y), np.abs(xx - x)).ravel()
    order = np.argsort(k, kind="stable")
    ks, vals = k[order], f.ravel()[order].astype(np.int64)
    starts = np.flatnonzero(np.r_[True, ks[1:] != ks[:-1]])
    ring_min = np.minimum.reduceat(vals, starts)
    return np.minimum.accumulate(ring_min)


def test_qdt_full_size_grey_sampled():
    f = synth.workload1_u8()["mask"]
    r, d, dl1 = run(f, 8)
    H, W = f.shape
    ys = RNG.integers(0, H, 40)
    xs = RNG.integers(0, W, 40)
    for y, x in zip(np.r_[ys, 0, H - 1, 0], np.r_[xs, 0, W - 1, W - 1]):
        e = ring_profile(f, y, x)
        res = e[:-1] - e[1:]
        rr = res.max() if res.size else 0
        dr = int(res.argmax()) + 1 if rr > 0 else 0
        assert r[y, x] == rr and d[y, x] == dr, (y, x)
    # d_l1: below d, 1-Lipschitz for the 3x3 neighbourhood, and the greatest such function
    assert np.all(dl1 <= d)
    assert np.abs(np.diff(dl1.astype(np.int64), axis=0)).max() <= 1
    assert np.abs(np.diff(dl1.astype(np.int64), axis=1)).max() <= 1
    assert np.abs(dl1[1:, 1:].astype(np.int64) - dl1[:-1, :-1]).max() <= 1
    assert np.abs(dl1[1:, :-1].astype(np.int64) - dl1[:-1, 1:]).max() <= 1
    yy, xx = np.mgrid[0:H, 0:W]
    for y, x in zip(ys[:12], xs[:12]):
        cheb = np.maximum(np.abs(yy - y), np.abs(xx - x))
        assert dl1[y, x] == (d.astype(np.int64) + cheb).min(), (y, x)


def test_qdt_full_size_binary_is_distance_transform():
    f = (RNG.random((1024, 1024)) < 0.999).astype(np.uint8) * 255
    r, d, dl1 = run(f, 8)
    np.testing.assert_array_equal(d, ndimage.distance_transform_cdt(f > 0, metric="chessboard"))
    np.testing.assert_array_equal(r, np.where(f > 0, 255, 0))
    np.testing.assert_array_equal(dl1, d)


def test_qdt_abi_in_place_lipschitz_and_errors():
    m = gm()
    lib = m.load()
    f = torch.from_numpy(synth.workload0(70, 90)["mask"]).cuda()
    r = torch.empty_like(f)
    d = torch.empty(f.shape, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    # d_l1 == d: the limit overwrites d
    assert lib.geo_qdt(0, f.data_ptr(), r.data_ptr(), d.data_ptr(), d.data_ptr(), 70, 90, 90, 8, s) == 0
    torch.cuda.synchronize()
    _, _, dlo = oracle.qdt(f.cpu().numpy(), 8)
    np.testing.assert_array_equal(d.cpu().numpy(), dlo)
    # d_l1 = NULL: part 1 only
    assert lib.geo_qdt(0, f.data_ptr(), r.data_ptr(), d.data_ptr(), None, 70, 90, 90, 8, s) == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d.cpu().numpy(), oracle.qdt_residual(f.cpu().numpy(), 8)[1])
    assert m.device_status() == 0
    # errors, all detected on the host before any work
    assert lib.geo_qdt(1, f.data_ptr(), r.data_ptr(), d.data_ptr(), None, 70, 90, 90, 8, s) == -2  # dtype
    assert lib.geo_qdt(0, f.data_ptr(), r.data_ptr(), d.data_ptr(), None, 70, 90, 80, 8, s) == -1  # pitch
    assert lib.geo_qdt(0, f.data_ptr(), r.data_ptr(), d.data_ptr(), None, 70, 90, 90, 6, s) == -1  # conn
    assert lib.geo_qdt(0, f.data_ptr(), r.data_ptr(), None, None, 70, 90, 90, 8, s) == -1  # no d
    assert lib.geo_qdt(0, f.data_ptr(), f.data_ptr(), d.data_ptr(), None, 70, 90, 90, 8, s) == -1  # r overlaps f
    assert lib.geo_qdt(0, f.data_ptr(), r.data_ptr(), d.data_ptr() + 2, None, 70, 90, 90, 8, s) == -3  # align
    assert lib.geo_qdt(0, f.data_ptr(), r.data_ptr(), d.data_ptr(), None, 1, 40000, 40000, 8, s) == -1  # S too long
    assert lib.geo_qdt(0, f.data_ptr(), r.data_ptr(), d.data_ptr(), None, 0, 90, 90, 8, s) == 0  # empty
