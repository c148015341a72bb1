"""GPU parity at the workloads' full sizes, in the launch configuration the
benchmark uses (the planners' default plans; for workload 3 also the
autotuned plans and the graph-captured batched launch the benchmark times).
Every output is compared with the SHA-256 of the oracle's output, written by
tests/golden/make_golden.py (which runs only the oracle):

* 1024x1024 (workload 1): every chain and window case.
* 4096x4096 (workload 2): the four reconstructions to stability (uint8 and
  float32 blob masks; the opening marker, the mask eroded by the 31x31
  square, and the h-dome marker mask - 20), and the opening marker itself.
  Beside the digests, properties that determine the result at any size are
  checked too: one more oracle step changes nothing (fixed point),
  marker <= out <= mask, and for sampled levels t the set {out >= t} is the
  union of the connected components of {mask >= t} that meet
  delta_1({marker >= t}) -- the least fixed point above the marker (Eq. 5).
* Workload 3 (512 items): every item of the batched launch, of the
  single-item calls and of the batched launch after autotuning.
"""
import hashlib
import json
import os

import numpy as np
import pytest
import torch
from scipy import ndimage

import oracle
import synth

pytestmark = pytest.mark.gpu

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
GOLDEN = os.path.join(GOLDEN_DIR, "workload1_sha256.json")
GOLDEN2 = os.path.join(GOLDEN_DIR, "workload2_sha256.json")
GOLDEN3 = os.path.join(GOLDEN_DIR, "workload3_sha256.json")


def gm():
    import paper_1911_13074_gb300 as m
    return m


def sha(t):
    torch.cuda.synchronize()
    return hashlib.sha256(np.ascontiguousarray(t.cpu().numpy()).tobytes()).hexdigest()


@pytest.mark.parametrize("f64_path", ["auto", "keys"])
def test_workload1_full_size_against_oracle_digests(f64_path, monkeypatch):
    """All 32 cases; float64 chains of 500 and 1500 steps take the rank
    transform by default, so they run once more on int64 keys."""
    if f64_path == "keys":
        monkeypatch.setenv("GEOMORPH_F64", "keys")
    cases = json.load(open(GOLDEN))["cases"]
    m = gm()
    data = {"u8": synth.workload1_u8(), "f64": synth.workload1_f64()}
    dev = {k: {n: torch.from_numpy(v).cuda() for n, v in w.items()} for k, w in data.items()}
    checked = 0
    for name, ref in cases.items():
        parts = name.split("_")
        if parts[0] == "chain":
            _, kind, op, conn, steps = parts
            conn, steps = int(conn[4:]), int(steps[5:])
            mk = dev[kind]["marker_dilate" if op == "dilate" else "marker_erode"]
            fn = m.dilate_chain if op == "dilate" else m.erode_chain
            out = fn(mk, dev[kind]["mask"], steps, conn=conn)
        else:
            _, kind, op, s = parts
            fn = m.window_dilate if op == "dilate" else m.window_erode
            out = fn(dev[kind]["mask"], int(s[1:]))
        assert sha(out) == ref["sha256"], f"{name}: output differs from the oracle's"
        checked += 1
    assert checked == 32
    assert m.device_status() == 0


def level_set_check(rec, marker, mask, conn, levels):
    st = ndimage.generate_binary_structure(2, 2 if conn == 8 else 1)
    for t in levels:
        M = mask >= t
        seeds = ndimage.binary_dilation(marker >= t, structure=st) & M
        lab, _ = ndimage.label(M, structure=st)
        keep = np.unique(lab[seeds])
        keep = keep[keep > 0]
        np.testing.assert_array_equal(rec >= t, np.isin(lab, keep), err_msg=f"level {t}")


@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_workload2_full_size_reconstruction(kind):
    w = synth.workload2()
    m = gm()
    digests = json.load(open(GOLDEN2))["cases"]
    mask = w["mask_u8"] if kind == "u8" else w["mask_f32"]
    hdome = w["hdome_marker_u8"] if kind == "u8" else w["hdome_marker_f32"]
    md = torch.from_numpy(mask).cuda()
    # (a) opening by reconstruction: marker = mask eroded by the 31x31 square
    ero = m.window_erode(md, 15)
    assert sha(ero) == digests[f"window_{kind}_erode_s15"]["sha256"], "31x31 erosion differs from the oracle's"
    ero_h = ero.cpu().numpy()
    for name, marker in (("open15", ero_h), ("hdome20", hdome)):
        rec, steps = m.reconstruct(torch.from_numpy(marker).cuda(), md, conn=8, return_steps=True)
        assert sha(rec) == digests[f"rec_{kind}_{name}_conn8"]["sha256"], f"{name}: differs from the oracle's"
        # the steps applied cover the oracle's changing steps plus the step that finds no change
        assert int(steps.item()) >= digests[f"rec_{kind}_{name}_conn8"]["oracle_changing_steps"] + 1
        out = rec.cpu().numpy()
        assert m.device_status() == 0
        assert np.all(marker <= out) and np.all(out <= mask)
        np.testing.assert_array_equal(oracle.step(out, mask, conn=8), out)  # fixed point
        levels = np.quantile(mask, [0.05, 0.2, 0.4, 0.6, 0.8, 0.9, 0.97, 0.995]).astype(mask.dtype)
        level_set_check(out, marker, mask, 8, np.unique(levels))


def test_workload3_every_item_against_oracle_digests():
    """The 512 items batched (the prepared launch captured in a CUDA graph and
    replayed, as the benchmark times it), as 512 single-item calls, and
    batched again after autotuning (the items' single-image plans, then the
    batch planner's policy on the batch itself): every output against its
    oracle digest."""
    m = gm()
    digests = json.load(open(GOLDEN3))["cases"]
    items = []
    for it in synth.workload3():
        items.append({"op": it["op"], "marker": torch.from_numpy(it["marker"]).cuda(),
                      "mask": torch.from_numpy(it["mask"]).cuda(),
                      "steps": 0 if it["steps"] < 0 else it["steps"], "conn": it["conn"]})

    def batched_graph():
        b = m.Batch(items).prepare()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            b.launch()
        torch.cuda.current_stream().wait_stream(s)
        for o in b.outs:
            o.fill_(7)  # what the replay writes is what is checked
        g.replay()
        b.check()
        return b.outs

    def compare(outs, what):
        bad = [i for i, o in enumerate(outs) if sha(o) != digests[f"item{i:03d}"]["sha256"]]
        assert not bad, f"{what}: items {bad[:10]} differ from the oracle ({len(bad)} of {len(outs)})"

    compare(batched_graph(), "batched (cost-model plans)")
    singles = []
    for it in items:
        op = it["op"]
        if op in (0, 1):
            singles.append((m.dilate_chain if op == 0 else m.erode_chain)(it["marker"], it["mask"], it["steps"],
                                                                        conn=it["conn"]))
        else:
            singles.append(m.reconstruct(it["marker"], it["mask"], conn=it["conn"],
                                         op="dilate" if op == 2 else "erode"))
    compare(singles, "single-item calls")
    try:
        m.autotune(items)
        m.Batch(items).autotune()
        compare(batched_graph(), "batched (autotuned plans)")
    finally:
        m.tune_reset()


def test_chain_and_window_past_32bit_offsets():
    """A 48000x48000 uint8 image (2.3e9 pixels, so byte offsets pass 2^31):
    a 6-step masked dilation chain and a 7x7 window dilation, checked on crops
    at the corners, the edges and the middle. A crop is computed by the oracle
    from the crop plus a halo as wide as the step count (or the image border),
    which fixes the crop exactly."""
    m = gm()
    H = W = 48000
    N, s = 6, 3
    gen = torch.Generator(device="cuda").manual_seed(0x6E0D00FF)
    mask = torch.randint(0, 256, (H, W), dtype=torch.uint8, device="cuda", generator=gen)
    marker = torch.clamp(mask, min=40) - 40  # saturating mask - 40
    out = m.dilate_chain(marker, mask, N, conn=8)
    win = m.window_dilate(mask, s)
    torch.cuda.synchronize()
    assert m.device_status() == 0
    C = 64
    for y0, x0 in [(0, 0), (0, W - C), (H - C, 0), (H - C, W - C), (H // 2 + 3, W // 2 - 5), (H - C, W // 3),
                   (46341, 46339)]:
        ya, yb = max(0, y0 - N), min(H, y0 + C + N)
        xa, xb = max(0, x0 - N), min(W, x0 + C + N)
        mk = marker[ya:yb, xa:xb].cpu().numpy()
        ms = mask[ya:yb, xa:xb].cpu().numpy()
        ref = oracle.chain(mk, ms, N, conn=8)[y0 - ya:y0 - ya + C, x0 - xa:x0 - xa + C]
        np.testing.assert_array_equal(out[y0:y0 + C, x0:x0 + C].cpu().numpy(), ref, err_msg=f"chain at {y0},{x0}")
        refw = oracle.window(ms, s)[y0 - ya:y0 - ya + C, x0 - xa:x0 - xa + C]
        np.testing.assert_array_equal(win[y0:y0 + C, x0:x0 + C].cpu().numpy(), refw, err_msg=f"window at {y0},{x0}")
    del mask, marker, out, win
    torch.cuda.empty_cache()
