"""GPU parity of the backward pass (reverse mode of the masked chain).

The CUDA gather sums gradients in the element type in a fixed order; the
oracle sums in float64. The bound per element is written relative to the
same backward run on |grad_out| (A(p), the sum of the magnitudes that reach
p), so cancellation in the signed sum cannot hide an error:
  |gpu - oracle| <= rtol * A(p),  rtol = 1e-12 (float64), 1e-5 (float32).
The routing decisions (argmax, tie rule, mask branch) are taken in the
element type on both sides (float32 values convert exactly to float64).
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

RTOL = {np.float32: 1e-5, np.float64: 1e-12}


def gm():
    import paper_1911_13074_gb300 as m
    return m


def oracle_batch(f, m, g, steps, conn, op):
    gmk = np.stack([oracle.chain_backward(f[b], m[b], g[b], steps, conn=conn, op=op)[0] for b in range(f.shape[0])])
    gms = np.stack([oracle.chain_backward(f[b], m[b], g[b], steps, conn=conn, op=op)[1] for b in range(f.shape[0])])
    a_mk = np.stack([oracle.chain_backward(f[b], m[b], np.abs(g[b]), steps, conn=conn, op=op)[0]
                     for b in range(f.shape[0])])
    a_ms = np.stack([oracle.chain_backward(f[b], m[b], np.abs(g[b]), steps, conn=conn, op=op)[1]
                     for b in range(f.shape[0])])
    return gmk, gms, a_mk, a_ms


def check_close(got, ref, scale, rtol, what):
    err = np.abs(got.astype(np.float64) - ref)
    bound = rtol * scale + 1e-300
    bad = err > bound
    if bad.any():
        i = np.argwhere(bad)[0]
        raise AssertionError(f"{what}: {bad.sum()} elements out of bound, first {tuple(i)}: "
                             f"gpu={got[tuple(i)]} oracle={ref[tuple(i)]} bound={bound[tuple(i)]}")


def run_case(B, H, W, dtype, steps, conn, op, C, seed):
    rng = np.random.default_rng(seed)
    m = rng.random((B, H, W)).astype(dtype)
    d = (0.2 * rng.random((B, H, W))).astype(dtype)
    f = (m - d if op == "dilate" else m + d).astype(dtype)
    g = rng.standard_normal((B, H, W)).astype(dtype)
    mod = gm()
    fm, mm, gg = (torch.from_numpy(x).cuda() for x in (f, m, g))
    out, ws = mod.chain_fwd_ckpt(fm, mm, steps, conn=conn, op=op, ckpt_interval=C)
    gmk, gms = mod.chain_backward(mm, gg, ws, steps, conn=conn, op=op, ckpt_interval=C)
    torch.cuda.synchronize()
    # forward output is bit-exact
    for b in range(B):
        np.testing.assert_array_equal(out[b].cpu().numpy(), oracle.chain(f[b], m[b], steps, conn=conn, op=op))
    ref_mk, ref_ms, a_mk, a_ms = oracle_batch(f, m, g, steps, conn, op)
    rt = RTOL[dtype]
    check_close(gmk.cpu().numpy(), ref_mk, a_mk, rt, f"grad_marker {dtype.__name__} {op} conn{conn} C={C}")
    check_close(gms.cpu().numpy(), ref_ms, a_ms, rt, f"grad_mask {dtype.__name__} {op} conn{conn} C={C}")
    # a second backward on the same workspace gives the same result
    gmk2, gms2 = mod.chain_backward(mm, gg, ws, steps, conn=conn, op=op, ckpt_interval=C)
    assert torch.equal(gmk, gmk2) and torch.equal(gms, gms2)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("op", ["dilate", "erode"])
@pytest.mark.parametrize("conn", [4, 8])
def test_backward_small_shapes(dtype, op, conn):
    for (B, H, W) in [(1, 1, 1), (2, 5, 7), (3, 37, 53)]:
        for steps, C in [(0, 4), (1, 1), (5, 2), (33, 16), (64, 64), (40, 64)]:
            run_case(B, H, W, dtype, steps, conn, op, C, seed=B * 1000 + steps)


@pytest.mark.parametrize("C", [16, 32, 64])
def test_backward_workload4_f32(C):
    """Workload 4 recipe (3x3-smoothed mask with jitter, marker = mask - U[0, 0.2]),
    8-connected 256-step dilation chain, float32, two images at the full 512x512."""
    w = synth.workload4(B=2, H=512, W=512)
    mod = gm()
    f, m, g = (torch.from_numpy(w[k]).cuda() for k in ("marker", "mask", "grad_out"))
    out, ws = mod.chain_fwd_ckpt(f, m, 256, conn=8, ckpt_interval=C)
    gmk, gms = mod.chain_backward(m, g, ws, 256, conn=8, ckpt_interval=C)
    torch.cuda.synchronize()
    for b in range(2):
        fb, mb, gb = w["marker"][b], w["mask"][b], w["grad_out"][b]
        np.testing.assert_array_equal(out[b].cpu().numpy(), oracle.chain(fb, mb, 256))
        rmk, rms = oracle.chain_backward(fb, mb, gb, 256)
        amk, ams = oracle.chain_backward(fb, mb, np.abs(gb), 256)
        check_close(gmk[b].cpu().numpy(), rmk, amk, 1e-5, f"workload4 grad_marker C={C}")
        check_close(gms[b].cpu().numpy(), rms, ams, 1e-5, f"workload4 grad_mask C={C}")


def test_backward_workload4_f64_autograd():
    """float64 at 64x64 through torch.autograd, against the oracle at 1e-12."""
    w = synth.workload4(B=3, H=64, W=64, dtype=np.float64)
    mod = gm()
    f = torch.from_numpy(w["marker"]).cuda().requires_grad_(True)
    m = torch.from_numpy(w["mask"]).cuda().requires_grad_(True)
    out = mod.geodesic_chain(f, m, 256, conn=8, ckpt_interval=32)
    out.backward(torch.from_numpy(w["grad_out"]).cuda())
    for b in range(3):
        rmk, rms = oracle.chain_backward(w["marker"][b], w["mask"][b], w["grad_out"][b], 256)
        amk, ams = oracle.chain_backward(w["marker"][b], w["mask"][b], np.abs(w["grad_out"][b]), 256)
        check_close(f.grad[b].cpu().numpy(), rmk, amk, 1e-12, "autograd grad_marker")
        check_close(m.grad[b].cpu().numpy(), rms, ams, 1e-12, "autograd grad_mask")


def test_backward_rejects_u8():
    mod = gm()
    lib = mod.load()
    assert lib.geo_chain_backward_workspace_size(0, 8, 8, 4, 2, 1) == 0
    x = torch.zeros(8, 8, dtype=torch.uint8, device="cuda")
    assert lib.geo_chain_fwd_ckpt(0, 0, x.data_ptr(), x.data_ptr(), x.data_ptr(), 8, 8, 8, 8, 4, 2, 1,
                                  x.data_ptr(), 64, None) == -2


def test_backward_workload4_full_batch_as_benchmarked():
    """The benchmark's launch configuration: all 32 images of workload 4 in
    one forward-with-checkpoints and one backward call (C = 16). Three
    images against the oracle; every image equal to a single-image call."""
    w = synth.workload4()
    mod = gm()
    f, m, g = (torch.from_numpy(w[k]).cuda() for k in ("marker", "mask", "grad_out"))
    out, ws = mod.chain_fwd_ckpt(f, m, 256, conn=8, ckpt_interval=16)
    gmk, gms = mod.chain_backward(m, g, ws, 256, conn=8, ckpt_interval=16)
    torch.cuda.synchronize()
    assert mod.device_status() == 0
    for b in (0, 13, 31):
        fb, mb, gb = w["marker"][b], w["mask"][b], w["grad_out"][b]
        np.testing.assert_array_equal(out[b].cpu().numpy(), oracle.chain(fb, mb, 256))
        rmk, rms = oracle.chain_backward(fb, mb, gb, 256)
        amk, ams = oracle.chain_backward(fb, mb, np.abs(gb), 256)
        check_close(gmk[b].cpu().numpy(), rmk, amk, 1e-5, f"batch image {b} grad_marker")
        check_close(gms[b].cpu().numpy(), rms, ams, 1e-5, f"batch image {b} grad_mask")
    for b in range(32):
        o1, ws1 = mod.chain_fwd_ckpt(f[b:b + 1], m[b:b + 1], 256, conn=8, ckpt_interval=16)
        k1, s1 = mod.chain_backward(m[b:b + 1], g[b:b + 1], ws1, 256, conn=8, ckpt_interval=16)
        assert torch.equal(o1[0], out[b]) and torch.equal(k1[0], gmk[b]) and torch.equal(s1[0], gms[b]), b
