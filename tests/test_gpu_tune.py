"""GPU checks of the autotuner: it measures (shape variant, K) per item,
persists the table (exact sizes and size classes), the planners use the
tuned plan, and results stay bit-exact against the oracle in every shape."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

# region (rows, columns) and threads per block of each shape variant
SHAPES = {torch.uint8: {0: (128, 128, 512), 1: (64, 128, 256), 2: (96, 128, 384)},
          torch.float32: {0: (128, 128, 512), 1: (64, 128, 256), 2: (64, 128, 512)}}


def gm():
    import paper_1911_13074_gb300 as m
    return m


@pytest.fixture(autouse=True)
def empty_tune_table():
    """Each test starts and ends with an empty tune table, so that no tuned
    plan reaches another test."""
    gm().tune_reset()
    yield
    gm().tune_reset()


def _pair(dtype, H, W, seed):
    w = synth.workload0(H, W, seed=seed)
    f, g = w["marker"], w["mask"]
    if dtype == torch.float32:
        f = (f.astype(np.float32) / np.float32(255)).astype(np.float32)
        g = (g.astype(np.float32) / np.float32(255)).astype(np.float32)
    return f, g


def test_autotune_persists_and_is_used(tmp_path):
    m = gm()
    w = synth.workload0(300, 260)
    f, g = torch.from_numpy(w["marker"]).cuda(), torch.from_numpy(w["mask"]).cuda()
    items = [{"op": "dilate_chain", "marker": f, "mask": g, "steps": 150, "conn": 8},
             {"op": "dilate_rec", "marker": f, "mask": g, "steps": 0, "conn": 4}]
    path = tmp_path / "tune.txt"
    m.autotune(items, path)
    lines = path.read_text().splitlines()
    assert lines[0].startswith("geomorph-tune 2 ")
    assert sum(ln.startswith("E ") for ln in lines) >= 2 and sum(ln.startswith("C ") for ln in lines) >= 2
    k_chain = m.tune_lookup(torch.uint8, "dilate_chain", 8, 300, 260, 150)
    k_rec = m.tune_lookup(torch.uint8, "dilate_rec", 4, 300, 260, 0)
    assert k_chain > 0 and k_rec > 0
    # the plan in force is the tuned (K, variant) of each entry
    entries = {}
    for ln in lines[1:]:
        p = ln.split()
        if p[0] == "E":
            entries[(int(p[2]), int(p[3]))] = (int(p[7]), int(p[8]), int(p[10]))
    K, TH, TW, v, thr = m.plan_shape(torch.uint8, "dilate_chain", 8, 300, 260, 150)
    assert (K, v) == entries[(0, 8)][:2]
    assert (TH + 2 * K, TW + 2 * K, thr) == SHAPES[torch.uint8][v]
    assert entries[(0, 8)][2] == k_chain  # the default-shape K the batch kernel uses
    K, TH, TW, v, thr = m.plan_shape(torch.uint8, "dilate_rec", 4, 300, 260, 0)
    assert (K, v) == entries[(2, 4)][:2]
    # the tuned plans compute the same results
    np.testing.assert_array_equal(m.dilate_chain(f, g, 150).cpu().numpy(),
                                  oracle.chain(w["marker"], w["mask"], 150))
    np.testing.assert_array_equal(m.reconstruct(f, g, conn=4).cpu().numpy(),
                                  oracle.reconstruct(w["marker"], w["mask"], conn=4)[0])
    # a reload of the file restores the same entries
    m.tune_load(path)
    assert m.tune_lookup(torch.uint8, "dilate_chain", 8, 300, 260, 150) == k_chain
    # another size in the same half-octave classes takes the class entry
    assert m.tune_lookup(torch.uint8, "dilate_chain", 8, 310, 270, 150) == k_chain


@pytest.mark.parametrize("dtype", [torch.uint8, torch.float32])
@pytest.mark.parametrize("variant", [1, 2])
def test_every_shape_variant_used_from_a_table_is_exact(dtype, variant, tmp_path):
    """A table naming a non-default shape (written here, loaded with
    geo_tune_load) is what the planner then uses, and every operation in that
    shape equals the oracle: chains of both operations and connectivities,
    reconstruction, and an in-place chain, on an image of several tiles with
    ragged edges."""
    m = gm()
    H, W = 211, 333
    f, g = _pair(dtype, H, W, 0x6E0D0200 + variant)
    dt = {torch.uint8: 0, torch.float32: 1}[dtype]
    K = 12
    path = tmp_path / "tune.txt"
    lines = ["geomorph-tune 2 test"]
    for op, conn, sc in [(0, 8, 64), (1, 4, 64), (2, 8, -1), (0, 4, 37)]:
        lines.append(f"E {dt} {op} {conn} {H} {W} {sc} {K} {variant} 1.0 {K} 1.0")
    path.write_text("\n".join(lines) + "\n")
    m.tune_load(path)
    rows, cols, thr = SHAPES[dtype][variant]
    for op, conn, steps in [("dilate_chain", 8, 150), ("erode_chain", 4, 90), ("dilate_rec", 8, 0)]:
        shape = m.plan_shape(dtype, op, conn, H, W, steps)
        assert shape == (K, rows - 2 * K, cols - 2 * K, variant, thr), (op, shape)
    mk, ms = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    # an erosion marker above the mask (the dual of the dilation marker)
    fe = (np.minimum(g.astype(np.int64) + 40, 255).astype(np.uint8) if dtype == torch.uint8
          else (g + np.float32(40.0 / 255.0)).astype(np.float32))
    np.testing.assert_array_equal(m.dilate_chain(mk, ms, 150).cpu().numpy(), oracle.chain(f, g, 150))
    np.testing.assert_array_equal(m.erode_chain(torch.from_numpy(fe).cuda(), ms, 90, conn=4).cpu().numpy(),
                                  oracle.chain(fe, g, 90, conn=4, op="erode"))
    np.testing.assert_array_equal(m.reconstruct(mk, ms).cpu().numpy(), oracle.reconstruct(f, g)[0])
    t = mk.clone()
    assert m.plan_shape(dtype, "dilate_chain", 4, H, W, 37)[3] == variant
    m.dilate_chain(t, ms, 37, conn=4, out=t)
    np.testing.assert_array_equal(t.cpu().numpy(), oracle.chain(f, g, 37, conn=4))


def test_tuner_chooses_and_uses_a_non_default_shape(tmp_path):
    """Images whose default-shape tiles leave most SMs idle (a narrow strip,
    small squares) run faster in the smaller regions of variants 1 and 2
    (more tiles, two blocks per SM for variant 1). The tuner measures every
    shape; at least one of these items ends with a non-default shape, which
    the planner then uses, persisted, and the result equals the oracle."""
    m = gm()
    cases = [(torch.uint8, 1000, 100), (torch.uint8, 180, 150), (torch.float32, 900, 120)]
    items, host = [], []
    for i, (dtype, H, W) in enumerate(cases):
        f, g = _pair(dtype, H, W, 0x6E0D0300 + i)
        items.append({"op": "dilate_chain", "marker": torch.from_numpy(f).cuda(),
                      "mask": torch.from_numpy(g).cuda(), "steps": 300, "conn": 8})
        host.append((dtype, H, W, f, g))
    path = tmp_path / "tune.txt"
    m.autotune(items, path)
    m.tune_load(path)
    chosen = []
    for (dtype, H, W, f, g), it in zip(host, items):
        K, TH, TW, v, thr = m.plan_shape(dtype, "dilate_chain", 8, H, W, 300)
        assert (TH + 2 * K, TW + 2 * K, thr) == SHAPES[dtype][v]
        chosen.append(v)
        np.testing.assert_array_equal(m.dilate_chain(it["marker"], it["mask"], 300).cpu().numpy(),
                                      oracle.chain(f, g, 300), err_msg=f"{dtype} {H}x{W} variant {v}")
    assert any(v != 0 for v in chosen), f"the tuner kept the default shape everywhere: {chosen}"
