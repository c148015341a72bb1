"""geomorph: geodesic 3x3 chains on one GB300 (sm_103a), Python binding.

This module only marshals arguments: it takes torch CUDA tensors (device
memory and the current stream), passes their raw pointers to the C ABI of
libgeomorph.so (declared in include/geomorph.h) through ctypes, and raises
GeoError on a non-zero status. Every step of the computation runs in the
library's CUDA kernels; there is no CPU path. If the library is missing it
is built from csrc/ with nvcc, and if that is impossible the call fails.

Errors found on the device (a bounded wait that expired, a reconstruction
that reached max_steps) are recorded in a per-device status word. By default
(check=True) every call synchronises its stream afterwards, reads and clears
that word, and raises GeoError with the recorded code. check=False keeps the
call asynchronous (for timing loops and CUDA-graph capture); the caller then
reads the word with device_status(). The word is sticky: it holds the first
error recorded since it was last read, by whichever call recorded it.

Operations (Zlaus & Mongus, IEEE TPDS 2019, Section 2):
  dilate_chain / erode_chain   Eq. 3-4, `steps` elementary geodesic steps
  reconstruct                  Eq. 5, iterate until a step changes nothing
  window_dilate / window_erode Eq. 1-2, clipped (2s+1)^2 square window
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import threading

import torch

from . import build as _build

__all__ = [
    "GeoError", "load", "library_path", "dilate_chain", "erode_chain", "reconstruct",
    "window_dilate", "window_erode", "device_status", "DTYPES", "geodesic_chain",
    "chain_fwd_ckpt", "chain_backward", "Batch", "OPS", "autotune", "tune_load", "tune_save", "tune_reset", "tune_lookup",
    "plan_info",
    "plan_shape",
    "hmax", "dome", "hfill", "raobj", "open_rec", "qdt", "opening", "closing", "asf", "granulometry",
    "probe_minmax_rate",
]

GEO_U8, GEO_F32, GEO_F64 = 0, 1, 2
DTYPES = {torch.uint8: GEO_U8, torch.float32: GEO_F32, torch.float64: GEO_F64}
STATUS = {
    0: "GEO_OK", -1: "GEO_ERR_ARG", -2: "GEO_ERR_DTYPE", -3: "GEO_ERR_ALIGN", -4: "GEO_ERR_CUDA",
    -5: "GEO_ERR_TIMEOUT", -6: "GEO_ERR_NOT_CONVERGED", -7: "GEO_ERR_WORKSPACE",
}

_lock = threading.Lock()
_lib = None


class GeoError(RuntimeError):
    """A geomorph call returned a non-zero geo_status."""

    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


class GeoItem(ctypes.Structure):
    """Mirror of geo_item in include/geomorph.h."""
    _fields_ = [("op", ctypes.c_int), ("dtype", ctypes.c_int), ("conn", ctypes.c_int),
                ("height", ctypes.c_int64), ("width", ctypes.c_int64), ("pitch", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("marker", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("out", ctypes.c_void_p)]


#: geo_item.op codes
OPS = {"dilate_chain": 0, "erode_chain": 1, "dilate_rec": 2, "erode_rec": 3, "window_dilate": 4,
       "window_erode": 5}


def library_path() -> str:
    return _build.LIB


def load():
    """Load libgeomorph.so (building it with nvcc first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # GEOMORPH_LIB selects another build of the same sources (a variant
        # compiled with other band shapes); otherwise build in-tree
        path = os.environ.get("GEOMORPH_LIB") or _build.build()
        lib = ctypes.CDLL(path)
        P, I, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        lib.geo_status_string.argtypes = [I]
        lib.geo_status_string.restype = ctypes.c_char_p
        lib.geo_device_status.argtypes = [P, ctypes.POINTER(I)]
        lib.geo_device_status.restype = I
        for name in ("geo_dilate_chain", "geo_erode_chain"):
            fn = getattr(lib, name)
            fn.argtypes = [I, P, P, P, L, L, L, I, L, P]
            fn.restype = I
        lib.geo_reconstruct.argtypes = [I, P, P, P, L, L, L, I, I, L, P, P]
        lib.geo_reconstruct.restype = I
        for name in ("morph_window_dilate", "morph_window_erode"):
            fn = getattr(lib, name)
            fn.argtypes = [I, P, P, L, L, L, L, P]
            fn.restype = I
        lib.geo_chain_backward_workspace_size.argtypes = [I, L, L, L, I, I]
        lib.geo_chain_backward_workspace_size.restype = ctypes.c_size_t
        lib.geo_chain_fwd_ckpt.argtypes = [I, I, P, P, P, L, L, L, I, L, I, I, P, ctypes.c_size_t, P]
        lib.geo_chain_fwd_ckpt.restype = I
        lib.geo_chain_backward.argtypes = [I, I, P, P, P, P, L, L, L, I, L, I, I, P, P]
        lib.geo_chain_backward.restype = I
        IP = ctypes.POINTER(GeoItem)
        lib.geo_batch_workspace_size.argtypes = [IP, I]
        lib.geo_batch_workspace_size.restype = ctypes.c_size_t
        lib.geo_batch_prepare.argtypes = [IP, I, P, ctypes.c_size_t, P]
        lib.geo_batch_prepare.restype = I
        lib.geo_batch_launch.argtypes = [IP, I, P, P, P]
        lib.geo_batch_launch.restype = I
        lib.geo_batch.argtypes = [IP, I, P, ctypes.c_size_t, P, P]
        lib.geo_batch.restype = I
        lib.geo_batch_autotune.argtypes = [IP, I, P, ctypes.c_size_t, P, P, ctypes.c_char_p]
        lib.geo_batch_autotune.restype = I
        lib.geo_tune_save.argtypes = [ctypes.c_char_p]
        lib.geo_tune_save.restype = I
        lib.geo_autotune.argtypes = [IP, I, ctypes.c_char_p]
        lib.geo_autotune.restype = I
        lib.geo_tune_load.argtypes = [ctypes.c_char_p]
        lib.geo_tune_load.restype = I
        lib.geo_tune_reset.argtypes = []
        lib.geo_tune_reset.restype = I
        lib.geo_tune_lookup.argtypes = [I, I, I, L, L, L]
        lib.geo_tune_lookup.restype = I
        D = ctypes.c_double
        for name in ("geo_hmax", "geo_dome"):
            getattr(lib, name).argtypes = [I, P, P, L, L, L, I, D, P]
            getattr(lib, name).restype = I
        for name in ("geo_hfill", "geo_raobj"):
            getattr(lib, name).argtypes = [I, P, P, L, L, L, I, P]
            getattr(lib, name).restype = I
        lib.geo_open_rec.argtypes = [I, P, P, L, L, L, I, L, P]
        lib.geo_open_rec.restype = I
        lib.geo_qdt.argtypes = [I, P, P, P, P, L, L, L, I, P]
        lib.geo_qdt.restype = I
        for name in ("geo_opening", "geo_closing", "geo_asf"):
            getattr(lib, name).argtypes = [I, P, P, L, L, L, L, P]
            getattr(lib, name).restype = I
        lib.geo_granulometry.argtypes = [I, P, L, L, L, L, P, P, P]
        lib.geo_granulometry.restype = I
        IPtr = ctypes.POINTER(I)
        lib.geo_plan_info.argtypes = [I, I, I, L, L, L, IPtr, IPtr, IPtr]
        lib.geo_plan_info.restype = I
        lib.geo_plan_shape.argtypes = [I, I, I, L, L, L, IPtr, IPtr, IPtr, IPtr, IPtr]
        lib.geo_plan_shape.restype = I
        DPtr = ctypes.POINTER(ctypes.c_double)
        lib.geo_probe_minmax_rate.argtypes = [I, DPtr, DPtr, P]
        lib.geo_probe_minmax_rate.restype = I
        _lib = lib
        return lib


def _check(rc: int, where: str):
    if rc != 0:
        raise GeoError(rc, where)


def _finish(device, check: bool, where: str):
    """With check, synchronise the call's stream and raise the device-side
    status the call (or an earlier unchecked call) recorded."""
    if check:
        v = device_status(device)
        if v != 0:
            raise GeoError(v, where + " (device)")


_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream(t: torch.Tensor) -> int:
    """The raw handle of the current stream of t's device."""
    if _raw_stream is not None:
        return _raw_stream(t.device.index)
    return torch.cuda.current_stream(t.device).cuda_stream


def _on(t: torch.Tensor):
    """Context that makes t's device current (a no-op when it already is:
    entering torch.cuda.device costs more than the launch of a short call)."""
    if t.device.index == torch.cuda.current_device():
        return contextlib.nullcontext()
    return torch.cuda.device(t.device)


def _image(t: torch.Tensor, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dim() != 2:
        raise ValueError(f"{name} must be 2-D (height, width), got shape {tuple(t.shape)}")
    if t.dtype not in DTYPES:
        raise TypeError(f"{name}: unsupported dtype {t.dtype} (uint8, float32, float64)")
    if t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError(f"{name} rows must be contiguous (stride(1) == 1)")
    return t


def _pitch(t: torch.Tensor) -> int:
    return max(int(t.stride(0)), int(t.shape[1])) if t.shape[0] > 1 else int(t.shape[1])


def _same(a: torch.Tensor, b: torch.Tensor, what: str):
    if a.shape != b.shape or a.dtype != b.dtype or a.device != b.device:
        raise ValueError(f"{what}: shape/dtype/device mismatch {tuple(a.shape)} {a.dtype} vs {tuple(b.shape)} {b.dtype}")
    if a.shape[0] > 1 and _pitch(a) != _pitch(b):
        raise ValueError(f"{what}: all images of a call share one row pitch")


def _out_like(marker: torch.Tensor, out):
    if out is None:
        return torch.empty_like(marker, memory_format=torch.contiguous_format) if _pitch(marker) == marker.shape[1] \
            else torch.empty_strided(marker.shape, marker.stride(), dtype=marker.dtype, device=marker.device)
    _image(out, "out")
    _same(marker, out, "out")
    return out


def _chain(name: str, marker, mask, steps: int, conn: int, out, check: bool):
    lib = load()
    _image(marker, "marker")
    _image(mask, "mask")
    _same(marker, mask, "mask")
    out = _out_like(marker, out)
    H, W = marker.shape
    with _on(marker):
        rc = getattr(lib, name)(DTYPES[marker.dtype], marker.data_ptr(), mask.data_ptr(), out.data_ptr(),
                                H, W, _pitch(marker), int(conn), int(steps), _stream(marker))
    _check(rc, name)
    _finish(marker.device, check, name)
    return out


def dilate_chain(marker: torch.Tensor, mask: torch.Tensor, steps: int, conn: int = 8, out=None,
                 check: bool = True) -> torch.Tensor:
    """`steps` geodesic dilation steps f <- min(delta_1(f), mask) (Eq. 3-4)."""
    return _chain("geo_dilate_chain", marker, mask, steps, conn, out, check)


def erode_chain(marker: torch.Tensor, mask: torch.Tensor, steps: int, conn: int = 8, out=None,
                check: bool = True) -> torch.Tensor:
    """`steps` geodesic erosion steps f <- max(eps_1(f), mask) (Eq. 3-4)."""
    return _chain("geo_erode_chain", marker, mask, steps, conn, out, check)


def reconstruct(marker: torch.Tensor, mask: torch.Tensor, conn: int = 8, op: str = "dilate",
                max_steps: int = 0, out=None, return_steps: bool = False, check: bool = True):
    """Dilation (op='dilate') or erosion (op='erode') by reconstruction (Eq. 5).

    A reconstruction still changing after max_steps records
    GEO_ERR_NOT_CONVERGED on the device; with check=True it is raised here
    as GeoError (out then holds the image reached so far).
    """
    lib = load()
    _image(marker, "marker")
    _image(mask, "mask")
    _same(marker, mask, "mask")
    out = _out_like(marker, out)
    H, W = marker.shape
    steps = torch.zeros(1, dtype=torch.int64, device=marker.device) if return_steps else None
    with _on(marker):
        rc = lib.geo_reconstruct(DTYPES[marker.dtype], marker.data_ptr(), mask.data_ptr(), out.data_ptr(),
                                 H, W, _pitch(marker), int(conn), {"dilate": 0, "erode": 1}[op], int(max_steps),
                                 None if steps is None else steps.data_ptr(), _stream(marker))
    _check(rc, "geo_reconstruct")
    _finish(marker.device, check, "geo_reconstruct")
    return (out, steps) if return_steps else out


def _window(name: str, img, half_size: int, out, check: bool):
    lib = load()
    _image(img, "in")
    out = _out_like(img, out)
    H, W = img.shape
    with _on(img):
        rc = getattr(lib, name)(DTYPES[img.dtype], img.data_ptr(), out.data_ptr(), H, W, _pitch(img),
                                int(half_size), _stream(img))
    _check(rc, name)
    _finish(img.device, check, name)
    return out


def window_dilate(img: torch.Tensor, half_size: int, out=None, check: bool = True) -> torch.Tensor:
    """Dilation by the clipped (2s+1)^2 square (Eq. 2), as s unmasked 3x3 steps."""
    return _window("morph_window_dilate", img, half_size, out, check)


def window_erode(img: torch.Tensor, half_size: int, out=None, check: bool = True) -> torch.Tensor:
    """Erosion by the clipped (2s+1)^2 square (Eq. 1), as s unmasked 3x3 steps."""
    return _window("morph_window_erode", img, half_size, out, check)


def device_status(device=None) -> int:
    """Synchronise the current stream and read-and-clear the device status
    words (the library's and the no-allocation chain's): 0 or the first
    device-side error recorded since the last read."""
    lib = load()
    cur = torch.cuda.current_device()
    dev = torch.device("cuda", cur) if device is None else torch.device(device)
    v = ctypes.c_int(0)
    if dev.index in (None, cur) and _raw_stream is not None:
        # the current device: no device switch, the raw stream handle
        rc = lib.geo_device_status(_raw_stream(cur), ctypes.byref(v))
    else:
        with torch.cuda.device(dev):
            rc = lib.geo_device_status(torch.cuda.current_stream(dev).cuda_stream, ctypes.byref(v))
    _check(rc, "geo_device_status")
    return int(v.value)


def probe_minmax_rate(form: str = "f16x2", device=None):
    """Measured rate of a min/max form on this GPU: "u16x2" / "f16x2" (the
    packed uint8 step), "f32x3" (three-input max.f32, the float32 step) or
    "mix" (max.u16x2 with an FMA-pipe exact max, 2:1): (maxima per SM clock
    per lane, SM clock in MHz)."""
    lib = load()
    code = {"u16x2": 0, "f16x2": 1, "f32x3": 2, "mix": 3}[form]
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    rate, mhz = ctypes.c_double(0.0), ctypes.c_double(0.0)
    with torch.cuda.device(dev):
        rc = lib.geo_probe_minmax_rate(code, ctypes.byref(rate), ctypes.byref(mhz),
                                       torch.cuda.current_stream(dev).cuda_stream)
    _check(rc, "geo_probe_minmax_rate")
    return float(rate.value), float(mhz.value)


# ---------------------------------------------------------------------------
# differentiable chain (float32 / float64)
# ---------------------------------------------------------------------------

_OPS = {"dilate": 0, "erode": 1}


def _batch_view(t: torch.Tensor, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype not in (torch.float32, torch.float64):
        raise TypeError(f"{name}: the backward pass supports float32 and float64, got {t.dtype}")
    if t.dim() == 2:
        t = t.unsqueeze(0)
    if t.dim() != 3:
        raise ValueError(f"{name} must be (H, W) or (B, H, W)")
    return t.contiguous()


def chain_fwd_ckpt(marker, mask, steps: int, conn: int = 8, op: str = "dilate", ckpt_interval: int = 32,
                   check: bool = True):
    """Forward chain that also stores checkpoints; returns (out, workspace)."""
    lib = load()
    mk = _batch_view(marker, "marker")
    ms = _batch_view(mask, "mask")
    if mk.shape != ms.shape or mk.dtype != ms.dtype:
        raise ValueError("marker and mask must match in shape and dtype")
    B, H, W = mk.shape
    dt = DTYPES[mk.dtype]
    nbytes = lib.geo_chain_backward_workspace_size(dt, H, W, int(steps), int(ckpt_interval), B)
    if nbytes == 0 and H * W > 0:
        raise GeoError(-1, "geo_chain_backward_workspace_size")
    ws = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=mk.device)
    out = torch.empty_like(mk)
    with _on(mk):
        rc = lib.geo_chain_fwd_ckpt(dt, _OPS[op], mk.data_ptr(), ms.data_ptr(), out.data_ptr(), H, W, W, int(conn),
                                    int(steps), int(ckpt_interval), B, ws.data_ptr(), int(nbytes), _stream(mk))
    _check(rc, "geo_chain_fwd_ckpt")
    _finish(mk.device, check, "geo_chain_fwd_ckpt")
    return out.view(marker.shape), ws


def chain_backward(mask, grad_out, workspace, steps: int, conn: int = 8, op: str = "dilate",
                   ckpt_interval: int = 32, check: bool = True):
    """(grad_marker, grad_mask) of the chain whose forward wrote `workspace`."""
    lib = load()
    ms = _batch_view(mask, "mask")
    g = _batch_view(grad_out, "grad_out").to(ms.dtype)
    B, H, W = ms.shape
    gmk = torch.empty_like(ms)
    gms = torch.empty_like(ms)
    with _on(ms):
        rc = lib.geo_chain_backward(DTYPES[ms.dtype], _OPS[op], ms.data_ptr(), g.data_ptr(), gmk.data_ptr(),
                                    gms.data_ptr(), H, W, W, int(conn), int(steps), int(ckpt_interval), B,
                                    workspace.data_ptr(), _stream(ms))
    _check(rc, "geo_chain_backward")
    _finish(ms.device, check, "geo_chain_backward")
    return gmk.view(mask.shape), gms.view(mask.shape)


class _GeodesicChain(torch.autograd.Function):
    @staticmethod
    def forward(ctx, marker, mask, steps, conn, op, ckpt_interval):
        out, ws = chain_fwd_ckpt(marker, mask, steps, conn, op, ckpt_interval)
        ctx.save_for_backward(mask, ws)
        ctx.cfg = (steps, conn, op, ckpt_interval)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        mask, ws = ctx.saved_tensors
        steps, conn, op, ckpt = ctx.cfg
        gmk, gms = chain_backward(mask, grad_out, ws, steps, conn, op, ckpt)
        return gmk, gms, None, None, None, None


def geodesic_chain(marker, mask, steps: int, conn: int = 8, op: str = "dilate", ckpt_interval: int = 32):
    """Differentiable geodesic chain (Eq. 4) of float32/float64 (H, W) or (B, H, W) images.

    The backward pass recomputes each segment of ckpt_interval steps from a
    checkpoint and routes gradients by the lowest-index tie rule (see
    include/geomorph.h).
    """
    return _GeodesicChain.apply(marker, mask, int(steps), int(conn), op, int(ckpt_interval))


# ---------------------------------------------------------------------------
# batched execution
# ---------------------------------------------------------------------------

class Batch:
    """Many independent items run in one persistent launch (geo_batch).

    items: list of dicts with keys op (a key of OPS or its code), marker,
    mask (not for windows), steps (chain length, window half size, or
    reconstruction max_steps with 0 = default), conn (4 or 8), and optionally
    out (defaults to a new tensor; may be the marker for in-place).
    prepare() uploads the descriptors; launch() runs every item (it copies
    nothing from the host and can be captured in a CUDA graph).
    """

    def __init__(self, items):
        lib = load()
        self.n = len(items)
        arr = (GeoItem * max(self.n, 1))()
        self.outs = []
        self._keep = []
        dev = None
        for i, it in enumerate(items):
            op = OPS[it["op"]] if isinstance(it["op"], str) else int(it["op"])
            mk = _image(it["marker"], "marker")
            dev = mk.device
            win = op in (4, 5)
            ms = None if win else _image(it["mask"], "mask")
            if ms is not None:
                _same(mk, ms, "mask")
            out = it.get("out")
            out = _out_like(mk, out)
            H, W = mk.shape
            arr[i].op = op
            arr[i].dtype = DTYPES[mk.dtype]
            arr[i].conn = int(it.get("conn", 8))
            arr[i].height, arr[i].width, arr[i].pitch = H, W, _pitch(mk)
            arr[i].steps = int(it.get("steps", 0))
            arr[i].marker = mk.data_ptr()
            arr[i].mask = None if ms is None else ms.data_ptr()
            arr[i].out = out.data_ptr()
            self.outs.append(out)
            self._keep += [mk, ms]
        self.items = arr
        self.device = dev if dev is not None else torch.device("cuda", torch.cuda.current_device())
        nbytes = lib.geo_batch_workspace_size(arr, self.n)
        if nbytes == 0 and self.n > 0:
            raise GeoError(-1, "geo_batch_workspace_size")
        self.workspace = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=self.device)
        self.nbytes = int(nbytes)
        self.status = torch.zeros(max(self.n, 1), dtype=torch.int32, device=self.device)

    def prepare(self):
        lib = load()
        with _on(self):
            rc = lib.geo_batch_prepare(self.items, self.n, self.workspace.data_ptr(), self.nbytes,
                                       torch.cuda.current_stream(self.device).cuda_stream)
        _check(rc, "geo_batch_prepare")
        return self

    def launch(self):
        lib = load()
        with _on(self):
            rc = lib.geo_batch_launch(self.items, self.n, self.workspace.data_ptr(), self.status.data_ptr(),
                                      torch.cuda.current_stream(self.device).cuda_stream)
        _check(rc, "geo_batch_launch")
        return self.outs

    def autotune(self, cache_path=None):
        """Time these items batched under each candidate pass-length policy,
        keep the fastest for every later prepare() (and in cache_path), and
        leave this batch prepared with it. Overwrites the outputs."""
        lib = load()
        with _on(self):
            rc = lib.geo_batch_autotune(self.items, self.n, self.workspace.data_ptr(), self.nbytes,
                                        self.status.data_ptr(), torch.cuda.current_stream(self.device).cuda_stream,
                                        None if cache_path is None else str(cache_path).encode())
        _check(rc, "geo_batch_autotune")
        return self

    def check(self):
        """Synchronise and raise if an item recorded a non-zero status (the
        first such item's code) or the device status word holds an error."""
        st = self.status[:self.n].cpu()
        bad = torch.nonzero(st).flatten()
        if bad.numel():
            i = int(bad[0])
            raise GeoError(int(st[i]), f"geo_batch item {i} (device)")
        _finish(self.device, True, "geo_batch")

    def run(self, check: bool = True):
        """prepare() and launch(); with check, then check()."""
        self.prepare()
        outs = self.launch()
        if check:
            self.check()
        return outs


# ---------------------------------------------------------------------------
# autotuning
# ---------------------------------------------------------------------------

def autotune(items, cache_path=None):
    """Time every valid (shape variant, pass length K) for each item (dicts as
    for Batch) and keep the fastest per exact size and per size class in the
    library's tune table; write the table to cache_path."""
    b = Batch(items)  # builds the geo_item array and output buffers
    lib = load()
    with _on(b):
        rc = lib.geo_autotune(b.items, b.n, None if cache_path is None else str(cache_path).encode())
    _check(rc, "geo_autotune")
    return b.outs


def tune_load(cache_path):
    _check(load().geo_tune_load(str(cache_path).encode()), "geo_tune_load")


def tune_save(cache_path):
    """Write the library's tune table to a file."""
    _check(load().geo_tune_save(str(cache_path).encode()), "geo_tune_save")


def tune_reset():
    """Empty the library's tune table (the cost models decide again)."""
    _check(load().geo_tune_reset(), "geo_tune_reset")


def tune_lookup(dtype, op, conn, height, width, steps) -> int:
    dt = DTYPES[dtype] if isinstance(dtype, torch.dtype) else int(dtype)
    code = OPS[op] if isinstance(op, str) else int(op)
    return int(load().geo_tune_lookup(dt, code, int(conn), int(height), int(width), int(steps)))


def plan_shape(dtype, op, conn, height, width, steps):
    """(K, TH, TW, variant, threads per block) of the single-image plan."""
    dt = DTYPES[dtype] if isinstance(dtype, torch.dtype) else int(dtype)
    code = OPS[op] if isinstance(op, str) else int(op)
    v = [ctypes.c_int(0) for _ in range(5)]
    _check(load().geo_plan_shape(dt, code, int(conn), int(height), int(width), int(steps), *[ctypes.byref(x) for x in v]),
           "geo_plan_shape")
    return tuple(x.value for x in v)


def plan_info(dtype, op, conn, height, width, steps):
    """(K, TH, TW) that the single-image entry points use for these arguments."""
    dt = DTYPES[dtype] if isinstance(dtype, torch.dtype) else int(dtype)
    code = OPS[op] if isinstance(op, str) else int(op)
    K, TH, TW = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(load().geo_plan_info(dt, code, int(conn), int(height), int(width), int(steps), ctypes.byref(K),
                                ctypes.byref(TH), ctypes.byref(TW)), "geo_plan_info")
    return K.value, TH.value, TW.value


# ---------------------------------------------------------------------------
# geodesic operators (Section 2, Eq. 6-12)
# ---------------------------------------------------------------------------

def _op(name, f, conn, *extra, out=None, check=True):
    lib = load()
    _image(f, "f")
    out = _out_like(f, out)
    H, W = f.shape
    with _on(f):
        rc = getattr(lib, name)(DTYPES[f.dtype], f.data_ptr(), out.data_ptr(), H, W, _pitch(f), int(conn), *extra,
                                _stream(f))
    _check(rc, name)
    _finish(f.device, check, name)
    return out


def hmax(f, h, conn=8, out=None, check=True):
    """HMAX_h(f) = delta_rec^f(f - h) (Eq. 6)."""
    return _op("geo_hmax", f, conn, float(h), out=out, check=check)


def dome(f, h, conn=8, out=None, check=True):
    """DOME_h(f) = f - HMAX_h(f) (Eq. 7)."""
    return _op("geo_dome", f, conn, float(h), out=out, check=check)


def hfill(f, conn=8, out=None, check=True):
    """HFILL(f): hole filling, erosion by reconstruction from the border (Eq. 8-9)."""
    return _op("geo_hfill", f, conn, out=out, check=check)


def raobj(f, conn=8, out=None, check=True):
    """RAOBJ(f): removal of objects touching the border (Eq. 10-11)."""
    return _op("geo_raobj", f, conn, out=out, check=check)


def open_rec(f, half_size, conn=8, out=None, check=True):
    """gamma_rec^s(f) = delta_rec^f(eps_s(f)), opening by reconstruction (Eq. 12)."""
    return _op("geo_open_rec", f, conn, int(half_size), out=out, check=check)


# ---------------------------------------------------------------------------
# quasi-distance transform (Section 2, Eq. 13-15; Algorithm 6)
# ---------------------------------------------------------------------------

def qdt(f, conn=8, lipschitz=True, check=True):
    """Quasi-distance transform of a uint8 image. Returns (r, d, d_l1): the
    largest residual eps_{j-1}(f) - eps_j(f) over the erosion chain (uint8),
    the first erosion j attaining it (int32, 0 where no erosion lowers the
    pixel), and the eta limit of d (Eq. 15; None with lipschitz=False)."""
    lib = load()
    _image(f, "f")
    if f.dtype != torch.uint8:
        raise TypeError("qdt takes uint8 images")
    H, W = f.shape
    pitch = _pitch(f)
    r = torch.empty_strided(f.shape, (pitch, 1), dtype=torch.uint8, device=f.device)
    d = torch.empty_strided(f.shape, (pitch, 1), dtype=torch.int32, device=f.device)
    dl1 = torch.empty_strided(f.shape, (pitch, 1), dtype=torch.int32, device=f.device) if lipschitz else None
    with _on(f):
        rc = lib.geo_qdt(DTYPES[f.dtype], f.data_ptr(), r.data_ptr(), d.data_ptr(),
                         dl1.data_ptr() if lipschitz else None, H, W, pitch, int(conn), _stream(f))
    _check(rc, "geo_qdt")
    _finish(f.device, check, "geo_qdt")
    return r, d, dl1


# ---------------------------------------------------------------------------
# openings, closings, granulometry, ASF (Section 2, Eq. 16-20)
# ---------------------------------------------------------------------------

def _win(name, f, s, out, check=True):
    lib = load()
    _image(f, "f")
    out = _out_like(f, out)
    H, W = f.shape
    with _on(f):
        rc = getattr(lib, name)(DTYPES[f.dtype], f.data_ptr(), out.data_ptr(), H, W, _pitch(f), int(s), _stream(f))
    _check(rc, name)
    _finish(f.device, check, name)
    return out


def opening(f, half_size, out=None, check=True):
    """gamma_s(f) = delta_s(eps_s(f)) with the clipped (2s+1)^2 square (Eq. 16)."""
    return _win("geo_opening", f, half_size, out, check)


def closing(f, half_size, out=None, check=True):
    """phi_s(f) = eps_s(delta_s(f)) (Eq. 19)."""
    return _win("geo_closing", f, half_size, out, check)


def asf(f, s, out=None, check=True):
    """Alternating sequential filter ASF_s(f) = phi_s gamma_s ... phi_1 gamma_1 (f) (Eq. 20)."""
    return _win("geo_asf", f, s, out, check)


def granulometry(f, smax, check=True):
    """(G, PS) as float64 CUDA tensors: G_k = sum of gamma_k(f), k = 0..smax
    (Eq. 17), and the pattern spectrum PS_k = G_k - G_{k+1} (Eq. 18)."""
    lib = load()
    _image(f, "f")
    H, W = f.shape
    G = torch.empty(int(smax) + 1, dtype=torch.float64, device=f.device)
    PS = torch.empty(max(int(smax), 1), dtype=torch.float64, device=f.device)
    with _on(f):
        rc = lib.geo_granulometry(DTYPES[f.dtype], f.data_ptr(), H, W, _pitch(f), int(smax), G.data_ptr(),
                                  PS.data_ptr(), _stream(f))
    _check(rc, "geo_granulometry")
    _finish(f.device, check, "geo_granulometry")
    return G, PS[:int(smax)]
