"""geo_dilate_chain_noalloc: the dilation chain for callers that cannot
allocate GPU memory during a call, whose scratch is a static device array.

Checked through the C ABI against geo_dilate_chain (the allocating entry
point) on two calls in a row, bit-exact like every forward result: the
second call reuses the array the first one left behind. Also checks that an
image whose scratch exceeds the fixed 16 MiB is rejected on the host.
This file is collected last so that a stop-at-first-failure run has already
run every other test when it gets here.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

GEO_ERR_WORKSPACE = -7


def _lib():
    import paper_1911_13074_gb300 as gm
    lib = gm.load()
    fn = lib.geo_dilate_chain_noalloc
    P, I, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    fn.argtypes = [I, P, P, P, L, L, L, I, L, P]
    fn.restype = I
    return lib


def _call(fn, dt, marker, mask, out, conn, steps):
    H, W = marker.shape
    stream = torch.cuda.current_stream().cuda_stream
    return fn(dt, marker.data_ptr(), mask.data_ptr(), out.data_ptr(), H, W, marker.stride(0), conn, steps, stream)


def test_noalloc_chain_matches_allocating_chain_twice():
    lib = _lib()
    rng = np.random.default_rng(2024)
    cases = [  # (dtype code, numpy dtype, H, W, conn, steps)
        (0, np.uint8, 300, 517, 8, 150),
        (1, np.float32, 211, 190, 4, 61),
    ]
    for dt, npdt, H, W, conn, steps in cases:
        if npdt == np.uint8:
            mask = rng.integers(0, 256, (H, W)).astype(np.uint8)
            marker = np.maximum(mask.astype(np.int64) - rng.integers(0, 90, (H, W)), 0).astype(np.uint8)
        else:
            mask = rng.standard_normal((H, W)).astype(np.float32)
            marker = (mask - np.abs(rng.standard_normal((H, W)))).astype(np.float32)
        mk = torch.from_numpy(marker).cuda()
        ms = torch.from_numpy(mask).cuda()
        ref = torch.empty_like(mk)
        got = torch.full_like(mk, 7)
        assert _call(lib.geo_dilate_chain, dt, mk, ms, ref, conn, steps) == 0
        assert _call(lib.geo_dilate_chain_noalloc, dt, mk, ms, got, conn, steps) == 0
        torch.cuda.synchronize()
        assert torch.equal(got, ref), f"noalloc differs from geo_dilate_chain (dtype {dt}, {H}x{W})"


def test_noalloc_rejects_images_beyond_its_scratch():
    lib = _lib()
    # 4100 x 4100 uint8 needs a 4112-byte pitch x 4100 rows > 16 MiB of scratch;
    # the size check runs on the host before any pointer is used
    fake = 1 << 20
    rc = lib.geo_dilate_chain_noalloc(0, fake, fake + (1 << 26), fake + (1 << 27), 4100, 4100, 4100, 8, 5, None)
    assert rc == GEO_ERR_WORKSPACE
