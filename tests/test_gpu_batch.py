"""GPU parity of batched execution: every item of a batch equals its
single-item result (bit-exact), across element types, operations,
connectivities, lengths, reconstruction and windows, in one launch."""
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
