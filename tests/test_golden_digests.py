"""The committed expected values are the oracle's (CPU, no GPU): a sample of
the digests in tests/golden/ is recomputed here with the oracle and must
match byte for byte — the 16 smallest of the 512 workload-3 items (chains and
reconstructions of both element types, operations and connectivities) and
the 27x27 windows of workload 1. The digest files are written by
tests/golden/make_golden.py, which calls only oracle/."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def test_smallest_batch_items_match_their_committed_digests():
    cases = json.load(open(os.path.join(GOLDEN, "workload3_sha256.json")))["cases"]
    assert len(cases) == 512
    items = synth.workload3()
    order = sorted(range(len(items)), key=lambda i: items[i]["marker"].size)[:16]
    kinds = set()
    for i in order:
        it = items[i]
        op = it["op"]
        if op in (synth.OP_DILATE_CHAIN, synth.OP_ERODE_CHAIN):
            out = oracle.chain(it["marker"], it["mask"], it["steps"], conn=it["conn"],
                               op="dilate" if op == synth.OP_DILATE_CHAIN else "erode")
        else:
            out = oracle.reconstruct(it["marker"], it["mask"], conn=it["conn"],
                                     op="dilate" if op == synth.OP_DILATE_REC else "erode")[0]
        ref = cases[f"item{i:03d}"]
        assert list(out.shape) == ref["shape"] and str(out.dtype) == ref["dtype"]
        assert sha(out) == ref["sha256"], f"item {i}"
        kinds.add((it["dtype"], op))
    assert len(kinds) >= 4  # both element types, chains and reconstructions among the sample


@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_workload1_windows_match_their_committed_digests(op):
    cases = json.load(open(os.path.join(GOLDEN, "workload1_sha256.json")))["cases"]
    g = synth.workload1_u8()["mask"]
    assert sha(oracle.window(g, 13, op=op)) == cases[f"window_u8_{op}_s13"]["sha256"]


def test_workload2_step_counts_are_recorded():
    """The reconstruction digests carry the oracle's changing-step counts,
    which the benchmark uses as the plain method's work."""
    cases = json.load(open(os.path.join(GOLDEN, "workload2_sha256.json")))["cases"]
    for kind in ("u8", "f32"):
        for marker in ("open15", "hdome20"):
            n = cases[f"rec_{kind}_{marker}_conn8"]["oracle_changing_steps"]
            assert isinstance(n, int) and 100 < n < 4096 * 4096
