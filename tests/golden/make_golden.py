"""Write tests/golden/workload1_sha256.json: digests of the CPU oracle's
outputs on the full-size 1024x1024 workload (uint8 and float64; dilation and
erosion chains of 100, 500 and 1500 steps at 4- and 8-connectivity; square
windows of half size 13 and 91). Only the oracle runs here; the GPU tests
compare the SHA-256 of the library's output bytes with these.

    python tests/golden/make_golden.py [--jobs N]
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload1_sha256.json")
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 4)
    a = ap.parse_args()
    import oracle
    oracle.build()
    chains = [(k, o, c) for k in ("u8", "f64") for o in ("dilate", "erode") for c in (4, 8)]
    wins = [(k, o, s) for k in ("u8", "f64") for o in ("dilate", "erode") for s in (13, 91)]
    ctx = mp.get_context("spawn")
    res = {}
    with ctx.Pool(a.jobs) as pool:
        for r in pool.imap_unordered(window_job, wins):
            res.update(r)
        for r in pool.imap_unordered(chain_job, chains):
            res.update(r)
    with open(OUT, "w") as fh:
        json.dump({"generator": "tests/golden/make_golden.py (CPU oracle, oracle/oracle.c)",
                   "workload": "synth.workload1_u8 / workload1_f64, 1024x1024, seed 0x6E0D0001",
                   "cases": dict(sorted(res.items()))}, fh, indent=1)
    print(f"wrote {len(res)} digests to {OUT}")


if __name__ == "__main__":
    main()
