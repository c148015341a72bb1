"""GPU parity of the geodesic operators (Eq. 6-12) against the oracle,
bit-exact, on random images up to 200x333 and the 256x256 workload-0 image.
The same operators on the 1024x1024 workload image the benchmark times
(Table 5's operators) are compared in full with oracle digests in
tests/test_gpu_table5_1024.py."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def gm():
    import paper_1911_13074_gb300 as m
    return m


def images(kind, rng):
    out = []
    for H, W in [(1, 1), (3, 70), (61, 45), (200, 333)]:
        if kind == "u8":
            out.append(rng.integers(0, 256, (H, W)).astype(np.uint8))
        else:
            out.append(rng.random((H, W)).astype(np.float32 if kind == "f32" else np.float64))
    w = synth.workload0()["mask"]
    out.append(w if kind == "u8" else (w.astype(np.float64) / 255).astype(np.float32 if kind == "f32" else np.float64))
    return out


@pytest.mark.parametrize("kind", ["u8", "f32", "f64"])
@pytest.mark.parametrize("conn", [4, 8])
def test_operators_match_oracle(kind, conn):
    m = gm()
    rng = np.random.default_rng(31 + conn)
    for f in images(kind, rng):
        h = 23 if kind == "u8" else 0.13
        t = torch.from_numpy(f).cuda()
        cases = [
            ("hmax", m.hmax(t, h, conn=conn), oracle.hmax(f, h, conn=conn)),
            ("dome", m.dome(t, h, conn=conn), oracle.dome(f, h, conn=conn)),
            ("hfill", m.hfill(t, conn=conn), oracle.hfill(f, conn=conn)),
            ("raobj", m.raobj(t, conn=conn), oracle.raobj(f, conn=conn)),
            ("open_rec", m.open_rec(t, 3, conn=conn), oracle.open_rec(f, 3, conn=conn)),
        ]
        for name, got, ref in cases:
            got = got.cpu().numpy()
            assert got.dtype == ref.dtype
            if not np.array_equal(got, ref):
                raise AssertionError(f"{name} {kind} conn{conn} {f.shape}: {(got != ref).sum()} mismatches")
    assert m.device_status() == 0


def test_operators_rejects_bad_arguments():
    m = gm()
    f = torch.zeros(8, 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(m.GeoError):
        m.hmax(f, -1.0)
    with pytest.raises(m.GeoError):
        m.hfill(f, out=f)  # out must not overlap f
