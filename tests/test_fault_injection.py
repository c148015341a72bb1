"""Failure reporting without faulting a GPU: GEOMORPH_FAULT injects the
failure on the host.

* badarg  — the call is rejected as an invalid argument before any CUDA work
            (runs without a GPU);
* alloc   — the scratch allocation fails: the call returns GEO_ERR_CUDA and
            the Python wrapper raises;
* timeout — the launch runs, but every wait on another CTA (the tagged words
            or neighbour epochs of a chain pass, the grid barrier of
            reconstruction) waits for something that never happens, expires
            after 20 ms and records
            GEO_ERR_TIMEOUT in the device status word; the kernel returns and
            the context stays usable (the next call is correct).
"""
import contextlib
import ctypes
import os

import numpy as np
import pytest

import oracle
import synth

GEO_ERR_ARG, GEO_ERR_CUDA, GEO_ERR_TIMEOUT = -1, -4, -5


def gm():
    import paper_1911_13074_gb300 as m
    return m


@contextlib.contextmanager
def fault(kind):
    os.environ["GEOMORPH_FAULT"] = kind
    try:
        yield
    finally:
        os.environ.pop("GEOMORPH_FAULT", None)


def test_badarg_is_rejected_on_the_host():
    lib = gm().load()
    p = ctypes.c_void_p(64)  # never dereferenced: the call returns first
    with fault("badarg"):
        assert lib.geo_dilate_chain(0, p, p, ctypes.c_void_p(4096), 8, 8, 8, 8, 5, None) == GEO_ERR_ARG
        assert lib.geo_reconstruct(1, p, p, ctypes.c_void_p(4096), 8, 8, 8, 8, 0, 0, None, None) == GEO_ERR_ARG
        assert lib.morph_window_erode(2, p, ctypes.c_void_p(4096), 8, 8, 8, 3, None) == GEO_ERR_ARG


@pytest.mark.gpu
def test_alloc_failure_raises():
    import torch
    m = gm()
    w = synth.workload0(64, 80)
    f, g = torch.from_numpy(w["marker"]).cuda(), torch.from_numpy(w["mask"]).cuda()
    with fault("alloc"):
        with pytest.raises(m.GeoError) as e:
            m.dilate_chain(f, g, 10)
    assert e.value.code == GEO_ERR_CUDA
    assert m.device_status() == 0
    np.testing.assert_array_equal(m.dilate_chain(f, g, 10).cpu().numpy(), oracle.chain(w["marker"], w["mask"], 10))


@pytest.mark.gpu
@pytest.mark.parametrize("kernel", ["rr", "rr-plain", "tile", "f64-ranks"])
def test_timeout_is_reported_and_the_context_stays_usable(kernel, monkeypatch):
    """f64-ranks: float64 on the rank path, whose chain and reconstruction
    hand over in rank-code words with a 7-bit pass tag (the injected wait is
    for a tag 64 passes away)."""
    import torch
    if kernel == "tile":
        monkeypatch.setenv("GEOMORPH_KERNEL", "tile")
    if kernel == "rr-plain":
        monkeypatch.setenv("GEOMORPH_TAGGED", "0")
    if kernel == "f64-ranks":
        monkeypatch.setenv("GEOMORPH_F64", "ranks")
    m = gm()
    w = synth.workload0(300, 300)
    if kernel == "f64-ranks":
        w = {k: v.astype(np.float64) for k, v in w.items()}
    f, g = torch.from_numpy(w["marker"]).cuda(), torch.from_numpy(w["mask"]).cuda()
    assert m.device_status() == 0
    with fault("timeout"):
        m.dilate_chain(f, g, 100, check=False)  # several passes: the neighbour waits expire
        assert m.device_status() == GEO_ERR_TIMEOUT
        m.reconstruct(f, g, check=False)  # the grid barrier expires
        assert m.device_status() == GEO_ERR_TIMEOUT
        # the checked form raises the same code at the call
        with pytest.raises(m.GeoError) as e:
            m.dilate_chain(f, g, 100)
        assert e.value.code == GEO_ERR_TIMEOUT
        with pytest.raises(m.GeoError) as e:
            m.reconstruct(f, g)
        assert e.value.code == GEO_ERR_TIMEOUT
    assert m.device_status() == 0
    np.testing.assert_array_equal(m.dilate_chain(f, g, 100).cpu().numpy(), oracle.chain(w["marker"], w["mask"], 100))
    np.testing.assert_array_equal(m.reconstruct(f, g).cpu().numpy(), oracle.reconstruct(w["marker"], w["mask"])[0])
    assert m.device_status() == 0
