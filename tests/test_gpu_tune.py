"""GPU checks of the autotuner: it measures K per item shape, persists the
table, the planners use the tuned K, and results stay bit-exact."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def gm():
    import paper_1911_13074_gb300 as m
    return m


def test_autotune_persists_and_is_used(tmp_path):
    m = gm()
    w = synth.workload0(300, 260)
    f, g = torch.from_numpy(w["marker"]).cuda(), torch.from_numpy(w["mask"]).cuda()
    items = [{"op": "dilate_chain", "marker": f, "mask": g, "steps": 150, "conn": 8},
             {"op": "dilate_rec", "marker": f, "mask": g, "steps": 0, "conn": 4}]
    path = tmp_path / "tune.txt"
    m.autotune(items, path)
    lines = path.read_text().splitlines()
    assert lines[0].startswith("geomorph-tune 1 ")
    assert len(lines) >= 3
    k_chain = m.tune_lookup(torch.uint8, "dilate_chain", 8, 300, 260, 150)
    k_rec = m.tune_lookup(torch.uint8, "dilate_rec", 4, 300, 260, 0)
    assert k_chain > 0 and k_rec > 0
    assert m.plan_info(torch.uint8, "dilate_chain", 8, 300, 260, 150)[0] == k_chain
    assert m.plan_info(torch.uint8, "dilate_rec", 4, 300, 260, 0)[0] == k_rec
    # the tuned plans compute the same results
    np.testing.assert_array_equal(m.dilate_chain(f, g, 150).cpu().numpy(),
                                  oracle.chain(w["marker"], w["mask"], 150))
    np.testing.assert_array_equal(m.reconstruct(f, g, conn=4).cpu().numpy(),
                                  oracle.reconstruct(w["marker"], w["mask"], conn=4)[0])
    # a reload of the file restores the same entries
    m.tune_load(path)
    assert m.tune_lookup(torch.uint8, "dilate_chain", 8, 300, 260, 150) == k_chain
