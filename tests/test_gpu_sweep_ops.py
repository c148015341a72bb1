"""Seeded sweep over the operator entry points (Section 2, Eq. 6-20) with
random shapes (sides 1 to 300, several tiles and ragged tails), element
types and connectivities, every result against the oracle (bit-exact; G_s
of float images within 1e-12 of the summed magnitudes)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

SIDES = [1, 2, 3, 7, 31, 33, 65, 100, 129, 200, 300]


def gm():
    import paper_1911_13074_gb300 as m
    return m


def image(rng, H, W, kind):
    g = synth.workload0(H, W, seed=int(rng.integers(1 << 30)))["mask"]
    if kind == "u8":
        return g
    x = g.astype(np.float64) / 255 + rng.normal(0, 1e-3, g.shape)
    return x.astype(np.float32 if kind == "f32" else np.float64)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def test_operator_sweep():
    m = gm()
    rng = np.random.default_rng(0x0F5EED)
    for case in range(18):
        H, W = int(rng.choice(SIDES)), int(rng.choice(SIDES))
        kind = ["u8", "f32", "f64"][case % 3]
        conn = 8 if case % 2 == 0 else 4
        f = image(rng, H, W, kind)
        fd = torch.from_numpy(f).cuda()
        h = 20 if kind == "u8" else 0.08
        what = f"case {case}: {kind} {H}x{W} conn{conn}"
        np.testing.assert_array_equal(host(m.hmax(fd, h, conn=conn)), oracle.hmax(f, h, conn=conn), err_msg=what)
        np.testing.assert_array_equal(host(m.dome(fd, h, conn=conn)), oracle.dome(f, h, conn=conn), err_msg=what)
        np.testing.assert_array_equal(host(m.hfill(fd, conn=conn)), oracle.hfill(f, conn=conn), err_msg=what)
        np.testing.assert_array_equal(host(m.raobj(fd, conn=conn)), oracle.raobj(f, conn=conn), err_msg=what)
        s = int(rng.integers(0, 6))
        np.testing.assert_array_equal(host(m.open_rec(fd, s, conn=conn)), oracle.open_rec(f, s, conn=conn),
                                      err_msg=what)
        np.testing.assert_array_equal(host(m.opening(fd, s)), oracle.opening(f, s), err_msg=what)
        np.testing.assert_array_equal(host(m.closing(fd, s)), oracle.closing(f, s), err_msg=what)
        np.testing.assert_array_equal(host(m.asf(fd, min(s, 3))), oracle.asf(f, min(s, 3)), err_msg=what)
        G, PS = m.granulometry(fd, 4)
        Go, PSo = oracle.granulometry(f, 4)
        tol = 0 if kind == "u8" else 1e-12 * np.abs(f.astype(np.float64)).sum()
        assert np.abs(host(G) - Go).max() <= tol and np.abs(host(PS) - PSo).max() <= 2 * tol, what
        if kind == "u8":
            r, d, dl1 = m.qdt(fd, conn=conn)
            ro, do_, dlo = oracle.qdt(f, conn)
            np.testing.assert_array_equal(host(r), ro, err_msg=what)
            np.testing.assert_array_equal(host(d), do_, err_msg=what)
            np.testing.assert_array_equal(host(dl1), dlo, err_msg=what)
    assert m.device_status() == 0
