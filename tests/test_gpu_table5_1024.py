"""The operators of the paper's Table 5 at the size the benchmark times them:
the 1024x1024 uint8 workload image, 8-connected, through the library's
default plans (the same calls bench.py makes). Every output byte is compared
with the SHA-256 of the oracle's output, written by tests/golden/make_golden.py
(which runs only the oracle):

* HMAX_20 and DOME_20 (Eq. 6-7), HFILL (Eq. 8-9), RAOBJ (Eq. 10-11) and the
  opening by reconstruction gamma_rec with s = 15 (Eq. 12): reconstructions
  to stability over many tiles and passes, where the skipping of settled
  tiles engages;
* the quasi-distance transform: r and d along the 1023-step erosion chain
  (Eq. 13, Algorithm 6) and the eta limit d_L1 (Eq. 14-15), every pixel.
"""
import hashlib
import json
import os

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table5_1024_sha256.json")


def sha(t):
    torch.cuda.synchronize()
    return hashlib.sha256(np.ascontiguousarray(t.cpu().numpy()).tobytes()).hexdigest()


@pytest.fixture(scope="module")
def image():
    return torch.from_numpy(synth.workload1_u8()["mask"]).cuda()


@pytest.fixture(scope="module")
def cases():
    return json.load(open(GOLDEN))["cases"]


@pytest.mark.parametrize("name", ["hmax_h20", "dome_h20", "hfill", "raobj", "open_rec_s15"])
def test_table5_operator_full_image_against_oracle_digest(name, image, cases):
    import paper_1911_13074_gb300 as gm
    fn = {"hmax_h20": lambda: gm.hmax(image, 20), "dome_h20": lambda: gm.dome(image, 20),
          "hfill": lambda: gm.hfill(image), "raobj": lambda: gm.raobj(image),
          "open_rec_s15": lambda: gm.open_rec(image, 15)}[name]
    out = fn()
    assert sha(out) == cases[f"{name}_conn8"]["sha256"], f"{name}: output differs from the oracle's"


def test_qdt_full_image_against_oracle_digest(image, cases):
    import paper_1911_13074_gb300 as gm
    r, d, dl1 = gm.qdt(image, conn=8)
    assert sha(r) == cases["qdt_r_conn8"]["sha256"], "qdt r differs from the oracle's"
    assert sha(d) == cases["qdt_d_conn8"]["sha256"], "qdt d differs from the oracle's"
    assert sha(dl1) == cases["qdt_dl1_conn8"]["sha256"], "qdt d_L1 differs from the oracle's"
