"""Write SHA-256 digests of the CPU oracle's outputs on the full-size
workloads. Only the oracle runs here; the GPU tests compare the SHA-256 of
the library's output bytes with these.

* set 1 -> workload1_sha256.json: the 1024x1024 workload (uint8 and float64;
  dilation and erosion chains of 100, 500 and 1500 steps at 4- and
  8-connectivity; square windows of half size 13 and 91).
* set 2 -> workload2_sha256.json: the four 4096x4096 reconstructions by
  dilation to stability (Eq. 5), uint8 and float32 blob masks, with the
  opening marker (the mask eroded by the 31x31 square, Eq. 1 and Eq. 12) and
  the h-dome marker (mask - 20, Eq. 6), 8-connected.
* set 3 -> workload3_sha256.json: every one of the 512 batched items (chains
  of Eq. 4 or reconstructions of Eq. 5, as drawn per item).
* set 4 -> table5_1024_sha256.json: the operators of the paper's Table 5 on
  the 1024x1024 uint8 workload image (the mask of set 1), 8-connected:
  HMAX_20 and DOME_20 (Eq. 6-7), HFILL (Eq. 8-9), RAOBJ (Eq. 10-11), the
  opening by reconstruction with s = 15 (Eq. 12), and the quasi-distance
  transform (r and d of Eq. 13 as Algorithm 6 computes them, and the eta
  limit of Eq. 14-15).

    python tests/golden/make_golden.py [--jobs N] [--sets 1,2,3,4]
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "workload1_sha256.json")
OUT2 = os.path.join(HERE, "workload2_sha256.json")
OUT3 = os.path.join(HERE, "workload3_sha256.json")
OUT4 = os.path.join(HERE, "table5_1024_sha256.json")
LENGTHS = (100, 500, 1500)


def digest(a):
    import numpy as np
    a = np.ascontiguousarray(a)
    return {"sha256": hashlib.sha256(a.tobytes()).hexdigest(), "shape": list(a.shape), "dtype": str(a.dtype)}


def chain_job(args):
    kind, op, conn = args
    import oracle
    import synth
    w = synth.workload1_u8() if kind == "u8" else synth.workload1_f64()
    f = w["marker_dilate"] if op == "dilate" else w["marker_erode"]
    out, done, res = f, 0, {}
    for n in LENGTHS:  # continue the same chain: chain(n) = chain(n - done) of chain(done)
        out = oracle.chain(out, w["mask"], n - done, conn=conn, op=op)
        done = n
        res[f"chain_{kind}_{op}_conn{conn}_steps{n}"] = digest(out)
    return res


def window_job(args):
    kind, op, s = args
    import oracle
    import synth
    w = synth.workload1_u8() if kind == "u8" else synth.workload1_f64()
    return {f"window_{kind}_{op}_s{s}": digest(oracle.window(w["mask"], s, op=op))}


def rec4096_job(args):
    kind, marker_kind = args
    import oracle
    import synth
    w = synth.workload2()
    mask = w["mask_u8"] if kind == "u8" else w["mask_f32"]
    if marker_kind == "open15":
        marker = oracle.window(mask, 15, op="erode")
    else:
        marker = w["hdome_marker_u8"] if kind == "u8" else w["hdome_marker_f32"]
    out, n = oracle.reconstruct(marker, mask, conn=8, op="dilate")
    d = digest(out)
    d["oracle_changing_steps"] = n
    res = {f"rec_{kind}_{marker_kind}_conn8": d}
    if marker_kind == "open15":
        res[f"window_{kind}_erode_s15"] = digest(marker)
    return res


def item_job(i):
    import oracle
    import synth
    it = synth.workload3()[i]
    op = it["op"]
    if op in (synth.OP_DILATE_CHAIN, synth.OP_ERODE_CHAIN):
        out = oracle.chain(it["marker"], it["mask"], it["steps"], conn=it["conn"],
                           op="dilate" if op == synth.OP_DILATE_CHAIN else "erode")
    else:
        out, _ = oracle.reconstruct(it["marker"], it["mask"], conn=it["conn"],
                                    op="dilate" if op == synth.OP_DILATE_REC else "erode")
    return i, digest(out)


def table5_job(name):
    import numpy as np
    import oracle
    import synth
    g = synth.workload1_u8()["mask"]
    if name == "qdt":
        r, d = oracle.qdt_residual(g, conn=8)
        dl1, _ = oracle.qdt_lipschitz(d, conn=8)
        return {"qdt_r_conn8": digest(r), "qdt_d_conn8": digest(d.astype(np.int32)),
                "qdt_dl1_conn8": digest(dl1.astype(np.int32))}
    fn = {"hmax_h20": lambda: oracle.hmax(g, 20, conn=8), "dome_h20": lambda: oracle.dome(g, 20, conn=8),
          "hfill": lambda: oracle.hfill(g, conn=8), "raobj": lambda: oracle.raobj(g, conn=8),
          "open_rec_s15": lambda: oracle.open_rec(g, 15, conn=8)}[name]
    return {f"{name}_conn8": digest(fn())}


def write(path, workload, res):
    with open(path, "w") as fh:
        json.dump({"generator": "tests/golden/make_golden.py (CPU oracle, oracle/oracle.c)",
                   "workload": workload, "cases": dict(sorted(res.items()))}, fh, indent=1)
    print(f"wrote {len(res)} digests to {path}", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 4)
    ap.add_argument("--sets", default="1,2,3")
    a = ap.parse_args()
    sets = {int(x) for x in a.sets.split(",") if x}
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.jobs) as pool:
        if 1 in sets:
            chains = [(k, o, c) for k in ("u8", "f64") for o in ("dilate", "erode") for c in (4, 8)]
            wins = [(k, o, s) for k in ("u8", "f64") for o in ("dilate", "erode") for s in (13, 91)]
            res = {}
            for r in pool.imap_unordered(window_job, wins):
                res.update(r)
            for r in pool.imap_unordered(chain_job, chains):
                res.update(r)
            write(OUT, "synth.workload1_u8 / workload1_f64, 1024x1024, seed 0x6E0D0001", res)
        pending4 = None
        if 4 in sets:
            pending4 = pool.map_async(table5_job, ["qdt", "hfill", "raobj", "open_rec_s15", "hmax_h20",
                                                   "dome_h20"])
        pending2 = None
        if 2 in sets:
            jobs = [(k, mk) for k in ("u8", "f32") for mk in ("open15", "hdome20")]
            pending2 = pool.map_async(rec4096_job, jobs)
        if 3 in sets:
            import synth
            items = synth.workload3()
            # largest first, so the long items do not finish last on one core
            order = sorted(range(len(items)), key=lambda i: -items[i]["marker"].size
                           * (4 if items[i]["steps"] < 0 else items[i]["steps"] / 500.0))
            del items
            res = {}
            for i, d in pool.imap_unordered(item_job, order):
                res[f"item{i:03d}"] = d
            write(OUT3, "synth.workload3, 512 items, seed 0x6E0D0003", res)
        if pending4 is not None:
            res = {}
            for r in pending4.get():
                res.update(r)
            write(OUT4, "synth.workload1_u8 mask, 1024x1024 uint8, seed 0x6E0D0001", res)
        if pending2 is not None:
            res = {}
            for r in pending2.get():
                res.update(r)
            write(OUT2, "synth.workload2, 4096x4096, seed 0x6E0D0002", res)


if __name__ == "__main__":
    main()
