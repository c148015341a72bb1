"""Single-image calls inside a CUDA graph: a chain and a reconstruction are
captured once (after a first call has set up the library's device state)
and replayed on new input data copied into the captured buffers; every
replay equals the oracle. The scratch comes from the stream-ordered pool,
which graph capture turns into graph memory nodes."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_chain_and_reconstruction_replay_in_a_graph():
    import paper_1911_13074_gb300 as m
    H, W = 200, 176
    inputs = [synth.workload0(H, W, seed=0x6E0D0100 + i) for i in range(3)]
    mk = torch.from_numpy(inputs[0]["marker"]).cuda()
    ms = torch.from_numpy(inputs[0]["mask"]).cuda()
    out_c = torch.empty_like(mk)
    out_r = torch.empty_like(mk)
    m.dilate_chain(mk, ms, 50, out=out_c)  # device state and plans exist before capture
    m.reconstruct(mk, ms, out=out_r)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        # no synchronising status read inside a capture: the asynchronous form
        m.dilate_chain(mk, ms, 50, out=out_c, check=False)
        m.reconstruct(mk, ms, out=out_r, check=False)
    for w in inputs[1:] + inputs[:1]:
        mk.copy_(torch.from_numpy(w["marker"]))
        ms.copy_(torch.from_numpy(w["mask"]))
        g.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out_c.cpu().numpy(), oracle.chain(w["marker"], w["mask"], 50))
        np.testing.assert_array_equal(out_r.cpu().numpy(), oracle.reconstruct(w["marker"], w["mask"])[0])
    assert m.device_status() == 0
