"""GPU parity of batched execution: every item of a batch equals its
single-item result (bit-exact), across element types, operations,
connectivities, lengths, reconstruction and windows, in one launch."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

OPNAME = {0: ("chain", "dilate"), 1: ("chain", "erode"), 2: ("rec", "dilate"), 3: ("rec", "erode"),
          4: ("win", "dilate"), 5: ("win", "erode")}


def gm():
    import paper_1911_13074_gb300 as m
    return m


def oracle_item(op, f, m, steps, conn):
    kind, o = OPNAME[op]
    if kind == "chain":
        return oracle.chain(f, m, steps, conn=conn, op=o)
    if kind == "rec":
        return oracle.reconstruct(f, m, conn=conn, op=o)[0]
    return oracle.window(f, steps, op=o)


def random_items(rng, n, max_side, max_steps):
    items, host = [], []
    for i in range(n):
        H = int(rng.integers(1, max_side + 1))
        W = int(rng.integers(1, max_side + 1))
        dt = [np.uint8, np.float32, np.float64][i % 3]
        op = int(rng.integers(0, 6))
        conn = int(rng.choice([4, 8]))
        steps = int(rng.integers(0, max_steps + 1))
        if dt == np.uint8:
            m = rng.integers(0, 256, (H, W)).astype(np.uint8)
            d = rng.integers(0, 60, (H, W))
            f = np.clip(m.astype(np.int64) + (d if op in (1, 3) else -d), 0, 255).astype(np.uint8)
        else:
            m = rng.standard_normal((H, W)).astype(dt)
            d = np.abs(rng.standard_normal((H, W))).astype(dt)
            f = (m + d if op in (1, 3) else m - d).astype(dt)
        if op in (2, 3):
            steps = 0
        items.append({"op": op, "marker": torch.from_numpy(f).cuda(), "mask": torch.from_numpy(m).cuda(),
                      "steps": steps, "conn": conn})
        host.append((op, f, m, steps, conn))
    return items, host


def check(batch, host):
    outs = batch.outs
    torch.cuda.synchronize()
    st = batch.status[:len(host)].cpu().numpy()
    assert np.all(st == 0), f"item status {st}"
    for i, (op, f, m, steps, conn) in enumerate(host):
        got = outs[i].cpu().numpy()
        ref = oracle_item(op, f, m, steps, conn)
        if not np.array_equal(got, ref):
            raise AssertionError(f"item {i} op={op} {f.dtype} {f.shape} steps={steps} conn={conn}: "
                                 f"{int((got != ref).sum())} mismatches")


def test_mixed_batch_matches_oracle():
    rng = np.random.default_rng(77)
    items, host = random_items(rng, 60, 300, 90)
    b = gm().Batch(items)
    b.run()
    check(b, host)
    assert gm().device_status() == 0


def test_batch_with_large_and_tiny_items():
    rng = np.random.default_rng(5)
    items, host = random_items(rng, 6, 700, 300)
    tiny, host_t = random_items(rng, 30, 3, 5)
    b = gm().Batch(items + tiny)
    b.run()
    check(b, host + host_t)


def test_empty_single_and_empty_items():
    m = gm()
    b = m.Batch([])
    b.run()
    x = torch.zeros((0, 5), dtype=torch.uint8, device="cuda")
    f = np.array([[3, 9], [1, 2]], np.uint8)
    g = np.array([[5, 9], [7, 2]], np.uint8)
    b = m.Batch([{"op": 0, "marker": x, "mask": x, "steps": 3},
                 {"op": 0, "marker": torch.from_numpy(f).cuda(), "mask": torch.from_numpy(g).cuda(), "steps": 1}])
    b.run()
    torch.cuda.synchronize()
    assert b.status[:2].tolist() == [0, 0]
    np.testing.assert_array_equal(b.outs[1].cpu().numpy(), oracle.chain(f, g, 1))


def test_in_place_items():
    rng = np.random.default_rng(9)
    items, host = random_items(rng, 12, 200, 70)
    for it in items:
        if it["op"] not in (4, 5):
            it["marker"] = it["marker"].clone()
            it["out"] = it["marker"]
    b = gm().Batch(items)
    b.run()
    check(b, host)


def test_graph_capture_and_replay():
    """Prepare once, capture the launch in a CUDA graph, replay it with new inputs."""
    rng = np.random.default_rng(13)
    items, host = random_items(rng, 20, 160, 60)
    b = gm().Batch(items).prepare()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.launch()
    for rep in range(2):
        # new inputs in the same buffers
        new_host = []
        for it, (op, f, m, steps, conn) in zip(items, host):
            f2 = f.copy()
            if f2.size:
                f2.flat[rep % f2.size] = f2.flat[0] if f2.dtype != np.uint8 else 0
            it["marker"].copy_(torch.from_numpy(f2))
            new_host.append((op, f2, m, steps, conn))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        check(b, new_host)


def test_workload3_sample_matches_single_item_calls():
    """Workload-3 generator (log-uniform sizes, W not a multiple of 32, half
    u8 / half f32, 25 % to stability) at reduced size: batched = oracle."""
    w = synth.workload3(n_items=48, lo=64, hi=384, max_steps=200)
    items, host = [], []
    for it in w:
        items.append({"op": it["op"], "marker": torch.from_numpy(it["marker"]).cuda(),
                      "mask": torch.from_numpy(it["mask"]).cuda(),
                      "steps": 0 if it["steps"] < 0 else it["steps"], "conn": it["conn"]})
        host.append((it["op"], it["marker"], it["mask"], 0 if it["steps"] < 0 else it["steps"], it["conn"]))
    b = gm().Batch(items)
    b.run()
    check(b, host)


def test_launch_captured_as_a_fresh_process_first_library_work():
    """In a process whose first library work is a batch, prepare() sets up
    the device state, so that the launch captured right after it allocates
    nothing inside the capture."""
    import subprocess
    import sys
    code = """
import numpy as np, torch, sys
sys.path.insert(0, %r)
import paper_1911_13074_gb300 as m, oracle, synth
w = synth.workload0(150, 170)
f, g = torch.from_numpy(w['marker']).cuda(), torch.from_numpy(w['mask']).cuda()
b = m.Batch([{'op': 'dilate_chain', 'marker': f, 'mask': g, 'steps': 40, 'conn': 8}]).prepare()
s = torch.cuda.Stream(); s.wait_stream(torch.cuda.current_stream())
gr = torch.cuda.CUDAGraph()
with torch.cuda.graph(gr, stream=s):
    b.launch()
torch.cuda.current_stream().wait_stream(s)
gr.replay(); b.check()
assert np.array_equal(b.outs[0].cpu().numpy(), oracle.chain(w['marker'], w['mask'], 40))
print('fresh-capture-ok')
""" % (os.path.dirname(os.path.dirname(os.path.abspath(__file__))),)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert "fresh-capture-ok" in r.stdout, r.stdout + r.stderr


def test_batch_autotune_persists_a_policy_and_stays_exact(tmp_path):
    """geo_batch_autotune times the batch under each candidate pass-length
    policy, keeps the fastest (written to the tune file as a B line), leaves
    the workspace prepared with it, and a new batch prepared afterwards uses
    it; every item still equals the oracle."""
    m = gm()
    m.tune_reset()
    try:
        rng = np.random.default_rng(31)
        items, host = random_items(rng, 24, 400, 300)
        b = m.Batch(items)
        path = tmp_path / "tune.txt"
        b.autotune(path)
        lines = path.read_text().splitlines()
        blines = [ln for ln in lines if ln.startswith("B ")]
        assert len(blines) == 1
        assert float(blines[0].split()[1]) in (2.5, 5.0, 10.0, 20.0, 40.0, 80.0)
        b.launch()
        check(b, host)
        b2 = m.Batch(items)
        b2.run()
        check(b2, host)
        m.tune_reset()
        m.tune_load(path)  # the policy comes back from the file
        b3 = m.Batch(items)
        b3.run()
        check(b3, host)
    finally:
        m.tune_reset()
