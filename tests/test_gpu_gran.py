"""GPU openings, closings, ASF and granulometry (Section 2, Eq. 16-20) against
the oracle, through the C ABI entry points geo_opening / geo_closing /
geo_asf / geo_granulometry.

Images compare element by element (bit-exact: the operators only select).
G_s is exact for uint8 images (integer sums in double); for float images the
GPU's fixed-order reduction and the oracle's row-by-row sum round
differently, so |G_gpu - G_oracle| <= 1e-12 * sum |f| is required.
At 1024x1024 (workload 1) the paper's Table 5 cases PS_[0,11] and ASF_11 run
in full against the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(1920)
SIZES = [(1, 1), (1, 37), (29, 1), (97, 131), (260, 301)]


def gm():
    import paper_1911_13074_gb300 as m
    return m


def img(H, W, kind):
    g = synth.workload0(H, W)["mask"]
    if kind == "u8":
        return g
    return (g.astype(np.float64) / 255 + RNG.normal(0, 1e-3, g.shape)).astype(np.float32 if kind == "f32" else np.float64)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("kind", ["u8", "u8-plain", "f32", "f64"])
@pytest.mark.parametrize("H,W", SIZES)
def test_opening_closing_asf_match_oracle(H, W, kind, monkeypatch):
    """uint8 programs of several tiles hand their passes over in tagged
    planes; "u8-plain" runs the same with plain planes and tile epochs."""
    if kind == "u8-plain":
        monkeypatch.setenv("GEOMORPH_TAGGED", "0")
        kind = "u8"
    m = gm()
    f = img(H, W, kind)
    fd = torch.from_numpy(f).cuda()
    for s in (0, 1, 3, 11):
        np.testing.assert_array_equal(host(m.opening(fd, s)), oracle.opening(f, s), err_msg=f"opening s={s}")
        np.testing.assert_array_equal(host(m.closing(fd, s)), oracle.closing(f, s), err_msg=f"closing s={s}")
    for s in (0, 1, 2, 5):
        np.testing.assert_array_equal(host(m.asf(fd, s)), oracle.asf(f, s), err_msg=f"asf s={s}")
    assert m.device_status() == 0


@pytest.mark.parametrize("kind", ["u8", "f32", "f64"])
@pytest.mark.parametrize("H,W", SIZES)
def test_granulometry_matches_oracle(H, W, kind):
    m = gm()
    f = img(H, W, kind)
    G, PS = m.granulometry(torch.from_numpy(f).cuda(), 6)
    Go, PSo = oracle.granulometry(f, 6)
    G, PS = host(G), host(PS)
    if kind == "u8":
        np.testing.assert_array_equal(G, Go)
        np.testing.assert_array_equal(PS, PSo)
    else:
        tol = 1e-12 * np.abs(f.astype(np.float64)).sum()
        assert np.abs(G - Go).max() <= tol and np.abs(PS - PSo).max() <= 2 * tol


@pytest.mark.parametrize("kind,smax", [("u8", 39), ("u8", 41), ("f64", 19), ("f64", 21), ("f32", 9)])
def test_granulometry_fused_sizes_and_fallback(kind, smax):
    """The granulometry runs one launch per size (erosion step, dilation
    steps and the per-tile sums together) while the halo (smax + 1, rounded
    up to whole lanes) fits a third of the register region's side (sizes up
    to 39 for uint8 and float32, 19 for float64), and the window calls
    beyond; both equal the oracle, on an image of many tiles with ragged
    edges."""
    m = gm()
    f = img(130, 150, kind)
    G, PS = m.granulometry(torch.from_numpy(f).cuda(), smax)
    Go, PSo = oracle.granulometry(f, smax)
    G, PS = host(G), host(PS)
    if kind == "u8":
        np.testing.assert_array_equal(G, Go)
        np.testing.assert_array_equal(PS, PSo)
    else:
        tol = 1e-12 * np.abs(f.astype(np.float64)).sum()
        assert np.abs(G - Go).max() <= tol and np.abs(PS - PSo).max() <= 2 * tol
    assert m.device_status() == 0


def test_in_place_and_pitched():
    m = gm()
    f = synth.workload0(150, 170)["mask"]
    big = torch.zeros((150, 200), dtype=torch.uint8, device="cuda")
    big[:, :170] = torch.from_numpy(f).cuda()
    view = big[:, :170]  # row pitch 200
    m.asf(view, 3, out=view)
    np.testing.assert_array_equal(host(view), oracle.asf(f, 3))
    assert not big[:, 170:].any()


def test_full_size_table5_cases():
    """PS_[0,11] and ASF_11 on the 1024x1024 workload-1 image."""
    m = gm()
    f = synth.workload1_u8()["mask"]
    fd = torch.from_numpy(f).cuda()
    G, PS = m.granulometry(fd, 11)
    Go, PSo = oracle.granulometry(f, 11)
    np.testing.assert_array_equal(host(G), Go)
    np.testing.assert_array_equal(host(PS), PSo)
    np.testing.assert_array_equal(host(m.asf(fd, 11)), oracle.asf(f, 11))
    assert m.device_status() == 0


def test_errors_detected_on_host():
    lib = gm().load()
    f = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    out = torch.zeros_like(f)
    G = torch.zeros(4, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.geo_opening(3, f.data_ptr(), out.data_ptr(), 8, 8, 8, 1, s) == -2
    assert lib.geo_asf(0, f.data_ptr(), out.data_ptr(), 8, 8, 7, 1, s) == -1
    assert lib.geo_closing(0, f.data_ptr(), f.data_ptr() + 1, 8, 8, 8, 1, s) == -1
    assert lib.geo_granulometry(0, f.data_ptr(), 8, 8, 8, 3, G.data_ptr() + 4, None, s) == -3
    assert lib.geo_granulometry(0, f.data_ptr(), 8, 8, 8, -1, G.data_ptr(), None, s) == -1
    assert lib.geo_granulometry(0, f.data_ptr(), 0, 8, 8, 3, G.data_ptr(), None, s) == 0
    torch.cuda.synchronize()
    assert not G.any()
