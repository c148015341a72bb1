"""GPU parity: the CUDA library against the CPU oracle, element by element.

Forward results only select among input values, so the bar is bit-exact
equality in every dtype. Inputs are seeded (synth/); expected values come
from the oracle only. Shapes span several tiles with ragged tails, single
rows and columns, and step counts around the pass length.
"""
import os
import zlib

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DEV = "cuda"


def gm():
    import paper_1911_13074_gb300 as m
    return m


@pytest.fixture(params=["rr", "rr-plain", "tile"])
def kernel(request, monkeypatch):
    """Run a test on the register-resident kernel (default: uint8 chains of
    one tile per CTA hand passes over in tagged planes), on the same kernel
    with plain planes and tile epochs (GEOMORPH_TAGGED=0), and on the
    shared-memory tile kernel (GEOMORPH_KERNEL=tile)."""
    monkeypatch.delenv("GEOMORPH_KERNEL", raising=False)
    monkeypatch.delenv("GEOMORPH_TAGGED", raising=False)
    if request.param == "tile":
        monkeypatch.setenv("GEOMORPH_KERNEL", "tile")
    elif request.param == "rr-plain":
        monkeypatch.setenv("GEOMORPH_TAGGED", "0")
    yield request.param


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rand_pair(H, W, kind, rng, op="dilate"):
    if kind == "u8":
        m = rng.integers(0, 256, (H, W)).astype(np.uint8)
        d = rng.integers(0, 80, (H, W))
        f = np.clip(m.astype(np.int64) + (d if op == "erode" else -d), 0, 255).astype(np.uint8)
    else:
        dt = np.float32 if kind == "f32" else np.float64
        m = rng.standard_normal((H, W)).astype(dt)
        d = np.abs(rng.standard_normal((H, W))).astype(dt)
        f = (m + d if op == "erode" else m - d).astype(dt)
    return f, m


def assert_same(got, ref, what=""):
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        y, x = bad[0]
        raise AssertionError(f"{what}: {len(bad)} mismatches, first at ({y},{x}): gpu={got[y, x]} oracle={ref[y, x]}")


SHAPES = [(1, 1), (1, 37), (29, 1), (3, 5), (17, 33), (64, 64), (100, 77), (129, 257), (250, 190)]


@pytest.mark.parametrize("kind", ["u8", "f32", "f64"])
@pytest.mark.parametrize("op", ["dilate", "erode"])
@pytest.mark.parametrize("conn", [4, 8])
def test_chain_parity_shapes_and_lengths(kind, op, conn, kernel):
    rng = np.random.default_rng(zlib.crc32(f"{kind} {op} {conn}".encode()))
    m = gm()
    fn = m.dilate_chain if op == "dilate" else m.erode_chain
    for H, W in SHAPES:
        f, msk = rand_pair(H, W, kind, rng, op)
        for steps in (0, 1, 2, 5, 11, 12, 13, 19, 20, 21, 23, 24, 25, 60):
            got = host(fn(dev(f), dev(msk), steps, conn=conn))
            ref = oracle.chain(f, msk, steps, conn=conn, op=op)
            assert_same(got, ref, f"{kind} {op} conn{conn} {H}x{W} steps={steps}")
    assert m.device_status() == 0


@pytest.mark.parametrize("kind", ["u8", "f32", "f64"])
@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_window_parity(kind, op, kernel):
    rng = np.random.default_rng(7)
    m = gm()
    fn = m.window_dilate if op == "dilate" else m.window_erode
    for H, W in [(1, 1), (7, 300), (300, 7), (131, 203)]:
        img = rand_pair(H, W, kind, rng)[1]
        for s in (0, 1, 4, 13, 40):
            got = host(fn(dev(img), s))
            assert_same(got, oracle.window(img, s, op), f"window {kind} {op} {H}x{W} s={s}")
            assert m.device_status() == 0, f"device status after window {kind} {op} {H}x{W} s={s}"


@pytest.mark.parametrize("kind", ["u8", "f32", "f64"])
@pytest.mark.parametrize("op", ["dilate", "erode"])
@pytest.mark.parametrize("conn", [4, 8])
def test_reconstruct_parity(kind, op, conn, kernel):
    rng = np.random.default_rng(11 + conn)
    m = gm()
    for H, W in [(1, 1), (1, 50), (40, 1), (45, 61), (150, 170)]:
        f, msk = rand_pair(H, W, kind, rng, op)
        assert m.device_status() == 0
        out, steps = m.reconstruct(dev(f), dev(msk), conn=conn, op=op, return_steps=True)
        ref, n = oracle.reconstruct(f, msk, conn=conn, op=op)
        assert_same(host(out), ref, f"rec {kind} {op} conn{conn} {H}x{W}")
        assert int(steps.item()) >= n
    assert m.device_status() == 0


def test_workload0_chain_and_reconstruction(kernel):
    """256x256 u8: 64-step 8-connected dilation chain, then reconstruction to stability."""
    w = synth.workload0()
    m = gm()
    f, msk = dev(w["marker"]), dev(w["mask"])
    assert_same(host(m.dilate_chain(f, msk, 64)), oracle.chain(w["marker"], w["mask"], 64), "chain64")
    rec, steps = m.reconstruct(f, msk, return_steps=True)
    ref, n = oracle.reconstruct(w["marker"], w["mask"])
    assert_same(host(rec), ref, "reconstruction")
    assert n > 0 and int(steps.item()) >= n
    assert m.device_status() == 0


@pytest.mark.parametrize("kind", ["u8", "f32", "f64"])
def test_in_place_and_strided(kind, kernel):
    rng = np.random.default_rng(3)
    m = gm()
    f, msk = rand_pair(90, 130, kind, rng)
    ref = oracle.chain(f, msk, 37)
    # in place: out aliases marker (odd and even pass counts)
    for steps in (37, 24, 1):
        t = dev(f)
        m.dilate_chain(t, dev(msk), steps, out=t)
        assert_same(host(t), oracle.chain(f, msk, steps), f"in-place {kind} steps={steps}")
    # row pitch larger than the width, odd (scalar path) and 16-byte multiple (vector path)
    for extra in (3, 16):
        big_f = dev(np.zeros((90, 135 + extra), f.dtype))
        big_m = dev(np.zeros((90, 135 + extra), f.dtype))
        big_o = dev(np.zeros((90, 135 + extra), f.dtype))
        vf, vm, vo = big_f[:, 5:135], big_m[:, 5:135], big_o[:, 5:135]
        vf.copy_(dev(f))
        vm.copy_(dev(msk))
        m.dilate_chain(vf, vm, 37, out=vo)
        assert_same(host(vo).copy(), ref, f"strided {kind} extra={extra}")
        # pixels outside the view are untouched
        assert np.all(host(big_o)[:, :5] == 0) and np.all(host(big_o)[:, 135:] == 0)


def test_reconstruct_not_converged_status():
    """A reconstruction capped below its chain length records
    GEO_ERR_NOT_CONVERGED on the device (Eq. 5 is not reached): the checked
    call raises it, the asynchronous call leaves it in the status word."""
    w = synth.workload0(64, 64)
    m = gm()
    with pytest.raises(m.GeoError) as e:
        m.reconstruct(dev(w["marker"]), dev(w["mask"]), max_steps=3)
    assert e.value.code == -6
    assert m.device_status() == 0  # the checked call read and cleared it
    m.reconstruct(dev(w["marker"]), dev(w["mask"]), max_steps=3, check=False)
    assert m.device_status() == -6
    assert m.device_status() == 0  # read clears
    # the same through an operator built on reconstruction, and a batch item
    out = m.reconstruct(dev(w["marker"]), dev(w["mask"]))  # converges: no error
    np.testing.assert_array_equal(host(out), oracle.reconstruct(w["marker"], w["mask"])[0])
    b = m.Batch([{"op": "dilate_rec", "marker": dev(w["marker"]), "mask": dev(w["mask"]), "steps": 3}])
    with pytest.raises(m.GeoError) as e:
        b.run()
    assert e.value.code == -6


def test_tagged_reconstruction_cap_and_step_count(monkeypatch):
    """uint8 reconstruction of several tiles (one per CTA) runs on tagged
    words with a per-pass vote instead of a grid barrier: the fixed point
    equals the oracle's, the steps it reports cover the oracle's changing
    steps plus the step that changes nothing, and capped below its length it
    records GEO_ERR_NOT_CONVERGED with out holding exactly the chain of the
    capped number of steps (each pass runs min(K, steps left))."""
    monkeypatch.delenv("GEOMORPH_TAGGED", raising=False)
    monkeypatch.delenv("GEOMORPH_KERNEL", raising=False)
    m = gm()
    w = synth.workload0(300, 420)
    f, msk = w["marker"], w["mask"]
    K, TH, TW = m.plan_info(torch.uint8, "dilate_rec", 8, 300, 420, 0)
    assert -(-300 // TH) * -(-420 // TW) >= 2  # several tiles
    out, steps = m.reconstruct(dev(f), dev(msk), return_steps=True)
    ref, n = oracle.reconstruct(f, msk)
    assert_same(host(out), ref, "tagged reconstruction")
    assert int(steps.item()) >= n + 1
    for cap in (37, 2 * K + 3):
        o = m.reconstruct(dev(f), dev(msk), max_steps=cap, check=False)
        assert m.device_status() == -6
        assert_same(host(o), oracle.chain(f, msk, cap), f"capped at {cap}")
    # erosion, in place, 4-connected
    e = np.minimum(msk.astype(np.int64) + 40, 255).astype(np.uint8)
    t = dev(e)
    m.reconstruct(t, dev(msk), conn=4, op="erode", out=t)
    assert_same(host(t), oracle.reconstruct(e, msk, conn=4, op="erode")[0], "tagged erosion, in place")
    assert m.device_status() == 0


def test_rank_code_reconstruction_cap_and_step_count(monkeypatch):
    """float64 reconstruction on the rank path: the float32 kernel runs on
    rank codes and, with several tiles (one per CTA), hands its passes over
    in 32-bit words that carry a 7-bit pass tag, with the per-pass vote
    instead of a grid barrier. The fixed point equals the oracle's, the
    reported steps cover the oracle's changing steps plus the step that
    changes nothing, and capped below its length it records
    GEO_ERR_NOT_CONVERGED with out holding exactly the chain of the capped
    number of steps."""
    monkeypatch.setenv("GEOMORPH_F64", "ranks")
    monkeypatch.delenv("GEOMORPH_TAGGED", raising=False)
    monkeypatch.delenv("GEOMORPH_KERNEL", raising=False)
    m = gm()
    w = synth.workload0(300, 420)
    rng = np.random.default_rng(0x7A6)
    msk = w["mask"].astype(np.float64) + np.round(rng.random((300, 420)) * 4.0) / 8.0  # ties and fractions
    f = np.minimum(w["marker"].astype(np.float64), msk)
    K, TH, TW = m.plan_info(torch.float32, "dilate_rec", 8, 300, 420, 0)
    assert -(-300 // TH) * -(-420 // TW) >= 2  # several tiles
    out, steps = m.reconstruct(dev(f), dev(msk), return_steps=True)
    ref, n = oracle.reconstruct(f, msk)
    assert_same(host(out), ref, "rank-code reconstruction")
    assert int(steps.item()) >= n + 1
    for cap in (37, 2 * K + 3):
        o = m.reconstruct(dev(f), dev(msk), max_steps=cap, check=False)
        assert m.device_status() == -6
        assert_same(host(o), oracle.chain(f, msk, cap), f"capped at {cap}")
    # erosion, in place, 4-connected
    e = msk + 40.0
    t = dev(e)
    m.reconstruct(t, dev(msk), conn=4, op="erode", out=t)
    assert_same(host(t), oracle.reconstruct(e, msk, conn=4, op="erode")[0], "rank-code erosion, in place")
    assert m.device_status() == 0


def test_full_size_1024_u8_chain(kernel):
    """1024x1024 u8 (workload 1), 100-step chains of both operations, whole image."""
    w = synth.workload1_u8()
    m = gm()
    for op, key in (("dilate", "marker_dilate"), ("erode", "marker_erode")):
        fn = m.dilate_chain if op == "dilate" else m.erode_chain
        got = host(fn(dev(w[key]), dev(w["mask"]), 100, conn=8))
        # full image for 100 steps
        assert_same(got, oracle.chain(w[key], w["mask"], 100, conn=8, op=op), f"1024 {op} 100")


def test_random_shape_sweep():
    """Seeded sweep: shapes with sides 1, 2, 3 and non-multiples of 4 / 16 /
    32 (including K larger than the image), every dtype, op and
    connectivity, chain lengths 0, 1, K - 1, K, K + 1 and 2K + 3 around the
    planned pass length K."""
    m = gm()
    rng = np.random.default_rng(0x5EED)
    sides = [1, 2, 3, 5, 7, 15, 31, 33, 47, 63, 65, 97, 131, 200, 301]
    for case in range(24):
        H, W = int(rng.choice(sides)), int(rng.choice(sides))
        kind = ["u8", "f32", "f64"][case % 3]
        op = "dilate" if (case // 3) % 2 == 0 else "erode"
        conn = 8 if (case // 6) % 2 == 0 else 4
        f, msk = rand_pair(H, W, kind, rng, op)
        dt = {"u8": torch.uint8, "f32": torch.float32, "f64": torch.float64}[kind]
        K, _, _ = m.plan_info(dt, op + "_chain", conn, H, W, 64)
        fn = m.dilate_chain if op == "dilate" else m.erode_chain
        for steps in sorted({0, 1, max(K - 1, 0), K, K + 1, 2 * K + 3}):
            got = host(fn(dev(f), dev(msk), steps, conn=conn))
            assert_same(got, oracle.chain(f, msk, steps, conn=conn, op=op),
                        f"{kind} {op} conn{conn} {H}x{W} K={K} steps={steps}")
    assert m.device_status() == 0


@pytest.mark.parametrize("H,W", [(300, 300), (129, 1000), (333, 517), (1024, 1024)])
def test_u8_tagged_hand_over(H, W):
    """uint8 chains of 3 and more passes with one tile per CTA hand the
    passes over in tagged planes: multi-tile shapes (a width not a multiple
    of 4 included), both ops and connectivities, 45 and 101 steps, in place."""
    m = gm()
    w = synth.workload0(H, W)
    f, msk = w["marker"], w["mask"]
    e = np.minimum(f.astype(np.int32) + 60, 255).astype(np.uint8)
    for conn in (4, 8):
        for steps in (45, 101):
            assert_same(host(m.dilate_chain(dev(f), dev(msk), steps, conn=conn)),
                        oracle.chain(f, msk, steps, conn=conn), f"dilate {H}x{W} conn{conn} {steps}")
            assert_same(host(m.erode_chain(dev(e), dev(msk), steps, conn=conn)),
                        oracle.chain(e, msk, steps, conn=conn, op="erode"), f"erode {H}x{W} conn{conn} {steps}")
            x = dev(f)
            m.dilate_chain(x, dev(msk), steps, conn=conn, out=x)
            assert_same(host(x), oracle.chain(f, msk, steps, conn=conn), f"in place {H}x{W} conn{conn} {steps}")
    assert m.device_status() == 0


@pytest.mark.parametrize("path", ["ranks", "keys"])
@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_f64_rank_and_key_paths(path, op, monkeypatch):
    """float64 long chains, windows and reconstructions run on the ranks of
    the values (an order isomorphism) or on int64 keys; both must equal the
    oracle bit for bit. Inputs mix many equal values, negative values and
    values a few ulps apart."""
    monkeypatch.setenv("GEOMORPH_F64", path)
    m = gm()
    rng = np.random.default_rng(0xF64)
    for H, W in [(1, 1), (1, 300), (37, 1), (130, 97), (257, 190)]:
        base = rng.integers(-40, 40, (H, W)).astype(np.float64) / 8.0      # many ties
        jit = np.where(rng.random((H, W)) < 0.3, np.spacing(base) * rng.integers(1, 4, (H, W)), 0.0)
        msk = base + jit
        d = np.abs(rng.standard_normal((H, W)))
        f = msk + d if op == "erode" else msk - d
        fn = m.dilate_chain if op == "dilate" else m.erode_chain
        for steps in (128, 200):
            assert_same(host(fn(dev(f), dev(msk), steps, conn=8)), oracle.chain(f, msk, steps, conn=8, op=op),
                        f"chain {path} {H}x{W} steps={steps}")
        win = m.window_dilate if op == "dilate" else m.window_erode
        assert_same(host(win(dev(msk), 130)), oracle.window(msk, 130, op=op), f"window {path} {H}x{W}")
        rec = host(m.reconstruct(dev(f), dev(msk), conn=4, op=op))
        assert_same(rec, oracle.reconstruct(f, msk, conn=4, op=op)[0], f"reconstruct {path} {H}x{W}")
        # in place, and rows with a pitch larger than the width
        t = dev(f)
        fn(t, dev(msk), 150, conn=8, out=t)
        assert_same(host(t), oracle.chain(f, msk, 150, conn=8, op=op), f"in place {path} {H}x{W}")
        big = torch.zeros((H, W + 5), dtype=torch.float64, device=DEV)
        big[:, :W] = dev(f)
        bm = torch.zeros_like(big)
        bm[:, :W] = dev(msk)
        o = fn(big[:, :W], bm[:, :W], 140, conn=8)
        assert_same(host(o), oracle.chain(f, msk, 140, conn=8, op=op), f"pitched {path} {H}x{W}")
    assert m.device_status() == 0
