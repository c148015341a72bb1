"""geo_dilate_chain_noalloc: the dilation chain for callers that cannot
allocate GPU memory during a call (a memory budget owned by another
allocator, a real-time loop that must not reach the driver's allocator),
whose scratch is a static device array.

Checked through the C ABI, bit-exact like every forward result, against
geo_dilate_chain (the allocating entry point) and against the oracle, on two
calls in a row per case: the second call reuses the array the first one left
behind. Covers uint8, float32 and float64, both connectivities, in-place
calls (marker == out) with odd and even pass counts, an injected timeout
that must be reported through geo_device_status, and an image whose scratch
exceeds the fixed 16 MiB, rejected on the host.
This file is collected last so that a stop-at-first-failure run has already
run every other test when it gets here.
"""
import contextlib
import ctypes
import os

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

GEO_ERR_TIMEOUT, GEO_ERR_WORKSPACE = -5, -7


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


def _status(lib):
    v = ctypes.c_int(0)
    assert lib.geo_device_status(torch.cuda.current_stream().cuda_stream, ctypes.byref(v)) == 0
    return v.value


def _inputs(rng, npdt, H, W):
    if npdt == np.uint8:
        mask = rng.integers(0, 256, (H, W)).astype(np.uint8)
        marker = np.maximum(mask.astype(np.int64) - rng.integers(0, 90, (H, W)), 0).astype(np.uint8)
    else:
        mask = rng.standard_normal((H, W)).astype(npdt)
        marker = (mask - np.abs(rng.standard_normal((H, W)))).astype(npdt)
    return marker, mask


CASES = [  # (dtype code, numpy dtype, H, W, conn, steps)
    (0, np.uint8, 300, 517, 8, 150),
    (1, np.float32, 211, 190, 4, 61),
    (2, np.float64, 150, 133, 8, 45),
]


@pytest.mark.parametrize("dt,npdt,H,W,conn,steps", CASES)
def test_noalloc_chain_matches_allocating_chain_and_oracle_twice(dt, npdt, H, W, conn, steps):
    lib = _lib()
    marker, mask = _inputs(np.random.default_rng(2024 + dt), npdt, H, W)
    want = oracle.chain(marker, mask, steps, conn=conn)
    mk = torch.from_numpy(marker).cuda()
    ms = torch.from_numpy(mask).cuda()
    ref = torch.empty_like(mk)
    assert _call(lib.geo_dilate_chain, dt, mk, ms, ref, conn, steps) == 0
    for call in range(2):  # the second call finds the first one's data in the shared array
        got = torch.full_like(mk, 7)
        assert _call(lib.geo_dilate_chain_noalloc, dt, mk, ms, got, conn, steps) == 0
        torch.cuda.synchronize()
        assert torch.equal(got, ref), f"call {call}: noalloc differs from geo_dilate_chain"
        np.testing.assert_array_equal(got.cpu().numpy(), want, err_msg=f"call {call}: noalloc differs from the oracle")
    assert _status(lib) == 0


@pytest.mark.parametrize("dt,npdt", [(0, np.uint8), (2, np.float64)])
def test_noalloc_in_place(dt, npdt):
    """out == marker: an odd pass count gets one more pass so that the first
    pass does not overwrite the image it reads; one step is always one pass."""
    lib = _lib()
    marker, mask = _inputs(np.random.default_rng(77 + dt), npdt, 181, 243)
    ms = torch.from_numpy(mask).cuda()
    for steps in (1, 37, 150):
        want = oracle.chain(marker, mask, steps, conn=8)
        ref = torch.empty(marker.shape, dtype=ms.dtype, device="cuda")
        assert _call(lib.geo_dilate_chain, dt, torch.from_numpy(marker).cuda(), ms, ref, 8, steps) == 0
        for call in range(2):
            t = torch.from_numpy(marker).cuda()
            assert _call(lib.geo_dilate_chain_noalloc, dt, t, ms, t, 8, steps) == 0
            torch.cuda.synchronize()
            assert torch.equal(t, ref), f"in place, steps {steps}, call {call}: differs from geo_dilate_chain"
            np.testing.assert_array_equal(t.cpu().numpy(), want, err_msg=f"in place, steps {steps}, call {call}")
    assert _status(lib) == 0


@contextlib.contextmanager
def _fault(kind):
    os.environ["GEOMORPH_FAULT"] = kind
    try:
        yield
    finally:
        os.environ.pop("GEOMORPH_FAULT", None)


def test_noalloc_timeout_is_reported_and_cleared():
    """Injected on the host: every wait on another block waits for a count
    that never comes, expires after 20 ms and records GEO_ERR_TIMEOUT in the
    array's status word. geo_device_status reports it (the word survives the
    next call's reset of the control words) and clears it; the next call is
    correct."""
    lib = _lib()
    marker, mask = _inputs(np.random.default_rng(9), np.uint8, 300, 300)
    mk = torch.from_numpy(marker).cuda()
    ms = torch.from_numpy(mask).cuda()
    out = torch.empty_like(mk)
    assert _status(lib) == 0
    with _fault("timeout"):
        assert _call(lib.geo_dilate_chain_noalloc, 0, mk, ms, out, 8, 100) == 0
        torch.cuda.synchronize()
    assert _call(lib.geo_dilate_chain_noalloc, 0, mk, ms, out, 8, 100) == 0  # a clean call in between
    assert _status(lib) == GEO_ERR_TIMEOUT
    assert _status(lib) == 0  # read clears
    assert _call(lib.geo_dilate_chain_noalloc, 0, mk, ms, out, 8, 100) == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.chain(marker, mask, 100, conn=8))
    assert _status(lib) == 0


def test_noalloc_rejects_images_beyond_its_scratch():
    lib = _lib()
    # 4100 x 4100 uint8 needs a 4112-byte pitch x 4100 rows > 16 MiB of scratch;
    # the size check runs on the host before any pointer is used
    fake = 1 << 20
    rc = lib.geo_dilate_chain_noalloc(0, fake, fake + (1 << 26), fake + (1 << 27), 4100, 4100, 4100, 8, 5, None)
    assert rc == GEO_ERR_WORKSPACE
