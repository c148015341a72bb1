"""Seeded synthetic inputs for the geodesic-chain workloads.

This module is shared by the CPU oracle tests, the GPU parity tests and the
benchmark. It only draws random numbers and shapes them into marker / mask
images; it contains none of the morphological arithmetic (no erosion,
dilation, geodesic step or reconstruction), so neither implementation can
inherit a mistake from it.

The paper evaluates on 1024x1024 photographs (Section 4, "Male", "Airport",
"Airplane"); those images are not available here, so every workload is a
synthetic stand-in with the same shape, dtype and value range.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): output i of a stream with key
k is mix(k + (i + 1) * 0x9E3779B97F4A7C15), evaluated vectorised in numpy
uint64 arithmetic (wrapping multiplication).
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

#: seed of workload c is SEED_BASE + c
SEED_BASE = 0x6E0D0000


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> int:
    """Key of an independent sub-stream (seed, stream) -> 64-bit key."""
    with np.errstate(over="ignore"):
        z = np.array([(seed * 0x100000001B3 + stream) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        return int(_mix(z + _GAMMA)[0])


def u64(seed: int, stream: int, n: int) -> np.ndarray:
    """n SplitMix64 outputs of sub-stream (seed, stream)."""
    key = np.uint64(stream_key(seed, stream))
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        return _mix(key + i * _GAMMA)


def uniform01(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles uniform on [0, 1) (top 53 bits)."""
    return (u64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal doubles by Box-Muller on two uniform streams."""
    u1 = 1.0 - uniform01(seed, 2 * stream + 1_000_001, n)  # (0, 1]
    u2 = uniform01(seed, 2 * stream + 1_000_002, n)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def uniform_int(seed: int, stream: int, n: int, lo: int, hi: int) -> np.ndarray:
    """n integers uniform on [lo, hi] (inclusive), by multiply-shift of the top 32 bits."""
    top = (u64(seed, stream, n) >> np.uint64(32)).astype(np.uint64)
    span = np.uint64(hi - lo + 1)
    return (lo + ((top * span) >> np.uint64(32)).astype(np.int64)).astype(np.int64)


def box_mean_u8(img: np.ndarray, radius: int) -> np.ndarray:
    """Clipped (2r+1)^2 box mean of a u8 image, rounded half up in integers.

    out = (2*sum + cnt) // (2*cnt) where sum and cnt run over the in-image
    part of the window. Used only to give the noise image spatial structure.
    """
    a = img.astype(np.int64)
    H, W = a.shape
    ii = np.zeros((H + 1, W + 1), np.int64)
    ii[1:, 1:] = a.cumsum(0).cumsum(1)
    y = np.arange(H)
    x = np.arange(W)
    y0 = np.clip(y - radius, 0, H)[:, None]
    y1 = np.clip(y + radius + 1, 0, H)[:, None]
    x0 = np.clip(x - radius, 0, W)[None, :]
    x1 = np.clip(x + radius + 1, 0, W)[None, :]
    s = ii[y1, x1] - ii[y0, x1] - ii[y1, x0] + ii[y0, x0]
    cnt = (y1 - y0) * (x1 - x0)
    return ((2 * s + cnt) // (2 * cnt)).astype(np.uint8)


def box_mean_f64(img: np.ndarray, radius: int) -> np.ndarray:
    """Clipped (2r+1)^2 box mean of a float image (float64)."""
    a = img.astype(np.float64)
    H, W = a.shape
    ii = np.zeros((H + 1, W + 1), np.float64)
    ii[1:, 1:] = a.cumsum(0).cumsum(1)
    y = np.arange(H)
    x = np.arange(W)
    y0 = np.clip(y - radius, 0, H)[:, None]
    y1 = np.clip(y + radius + 1, 0, H)[:, None]
    x0 = np.clip(x - radius, 0, W)[None, :]
    x1 = np.clip(x + radius + 1, 0, W)[None, :]
    s = ii[y1, x1] - ii[y0, x1] - ii[y1, x0] + ii[y0, x0]
    cnt = (y1 - y0) * (x1 - x0)
    return s / cnt


def textured_u8(seed: int, H: int, W: int, stream: int = 0) -> np.ndarray:
    """Workload-0 image g: clipped 5x5 box mean of i.i.d. uniform {0..255} noise."""
    noise = (u64(seed, stream, H * W) >> np.uint64(56)).astype(np.uint8).reshape(H, W)
    return box_mean_u8(noise, 2)


def sat_sub_u8(a: np.ndarray, c: int) -> np.ndarray:
    """Saturating a - c on u8 (input preparation, not a morphological step)."""
    return np.maximum(a.astype(np.int64) - c, 0).astype(np.uint8)


def sat_add_u8(a: np.ndarray, c: int) -> np.ndarray:
    return np.minimum(a.astype(np.int64) + c, 255).astype(np.uint8)


# ----------------------------------------------------------------------------
# Workloads. Each returns plain numpy arrays (C-contiguous, row-major).
# ----------------------------------------------------------------------------

def workload0(H: int = 256, W: int = 256, seed: int = SEED_BASE + 0):
    """256x256 u8 pair: mask g = 5x5 box blur of uniform noise, marker = max(g-40, 0)."""
    g = textured_u8(seed, H, W)
    return {"mask": g, "marker": sat_sub_u8(g, 40)}


def workload1_u8(H: int = 1024, W: int = 1024, seed: int = SEED_BASE + 1):
    """1024x1024 u8: mask g, dilation marker max(g-40,0), erosion marker min(g+40,255)."""
    g = textured_u8(seed, H, W)
    return {"mask": g, "marker_dilate": sat_sub_u8(g, 40), "marker_erode": sat_add_u8(g, 40)}


def workload1_f64(H: int = 1024, W: int = 1024, seed: int = SEED_BASE + 1):
    """1024x1024 f64: the u8 workload / 255 plus independent N(0, 1e-3) jitter.

    Where the jitter puts a dilation marker above the mask (or an erosion
    marker below it) the marker is set to the mask there, so that every pair
    satisfies marker <= mask (dilation) / marker >= mask (erosion).
    """
    w = workload1_u8(H, W, seed)
    n = H * W
    mask = w["mask"].astype(np.float64) / 255.0 + 1e-3 * normal(seed, 11, n).reshape(H, W)
    md = w["marker_dilate"].astype(np.float64) / 255.0 + 1e-3 * normal(seed, 12, n).reshape(H, W)
    me = w["marker_erode"].astype(np.float64) / 255.0 + 1e-3 * normal(seed, 13, n).reshape(H, W)
    md = np.minimum(md, mask)
    me = np.maximum(me, mask)
    return {"mask": mask, "marker_dilate": md, "marker_erode": me}


def blobs_f64(H: int, W: int, seed: int, n_blobs: int = 200) -> np.ndarray:
    """Sum of isotropic Gaussian blobs plus U[0,10) noise, clamped to [0, 255].

    Centre uniform over the image, sigma ~ U[5, 80] px, amplitude ~ U[20, 200].
    Each blob is evaluated within +-4 sigma of its centre (beyond that it is
    below 200 * exp(-8) < 0.07 and is left out).
    """
    cy = uniform01(seed, 21, n_blobs) * H
    cx = uniform01(seed, 22, n_blobs) * W
    sig = 5.0 + 75.0 * uniform01(seed, 23, n_blobs)
    amp = 20.0 + 180.0 * uniform01(seed, 24, n_blobs)
    out = np.zeros((H, W), np.float64)
    for b in range(n_blobs):
        r = int(np.ceil(4.0 * sig[b]))
        y0, y1 = max(0, int(cy[b]) - r), min(H, int(cy[b]) + r + 1)
        x0, x1 = max(0, int(cx[b]) - r), min(W, int(cx[b]) + r + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        yy = (np.arange(y0, y1) + 0.5 - cy[b])[:, None]
        xx = (np.arange(x0, x1) + 0.5 - cx[b])[None, :]
        out[y0:y1, x0:x1] += amp[b] * np.exp(-(yy * yy + xx * xx) / (2.0 * sig[b] * sig[b]))
    out += 10.0 * uniform01(seed, 25, H * W).reshape(H, W)
    return np.clip(out, 0.0, 255.0)


def workload2(H: int = 4096, W: int = 4096, seed: int = SEED_BASE + 2):
    """4096x4096 blob masks (u8 = round half up, f32 = unrounded) and the h-dome markers mask-20.

    The opening-by-reconstruction marker (mask eroded by a 31x31 square) is a
    morphological result, so each side computes it with its own window code.
    """
    m = blobs_f64(H, W, seed)
    mask_u8 = np.floor(m + 0.5).astype(np.uint8)
    mask_f32 = m.astype(np.float32)
    return {
        "mask_u8": mask_u8,
        "mask_f32": mask_f32,
        "hdome_marker_u8": sat_sub_u8(mask_u8, 20),
        "hdome_marker_f32": (mask_f32 - np.float32(20.0)).astype(np.float32),
    }


#: item op codes shared with the C ABI's geo_item.op
OP_DILATE_CHAIN, OP_ERODE_CHAIN, OP_DILATE_REC, OP_ERODE_REC, OP_WINDOW_DILATE, OP_WINDOW_ERODE = range(6)


def workload3(n_items: int = 512, lo: int = 64, hi: int = 2048, max_steps: int = 1500,
              seed: int = SEED_BASE + 3):
    """Batched workload: n items with log-uniform H, W in [lo, hi] (W not a multiple of 32).

    The first half are u8, the second half f32 (= u8 / 255). Chain length is
    uniform on {8..max_steps}; a quarter of the items (drawn) run to stability
    instead. Operation (dilate / erode) and connectivity (4 / 8) are drawn per
    item; erosion items use the dual marker min(g + 40, 255).
    Returns a list of dicts with keys op, dtype, conn, steps (-1 = to
    stability), marker, mask.
    """
    lh = np.log(lo) + (np.log(hi) - np.log(lo)) * uniform01(seed, 31, n_items)
    lw = np.log(lo) + (np.log(hi) - np.log(lo)) * uniform01(seed, 32, n_items)
    Hs = np.clip(np.rint(np.exp(lh)).astype(np.int64), lo, hi)
    Ws = np.clip(np.rint(np.exp(lw)).astype(np.int64), lo, hi)
    Ws = np.where(Ws % 32 == 0, Ws + np.where(Ws < hi, 1, -1), Ws)
    steps = uniform_int(seed, 33, n_items, 8, max_steps)
    to_stab = uniform01(seed, 34, n_items) < 0.25
    erode = uniform01(seed, 35, n_items) < 0.5
    conn8 = uniform01(seed, 36, n_items) < 0.5
    items = []
    for i in range(n_items):
        H, W = int(Hs[i]), int(Ws[i])
        g = textured_u8(seed, H, W, stream=1000 + i)
        if erode[i]:
            marker = sat_add_u8(g, 40)
            op = OP_ERODE_REC if to_stab[i] else OP_ERODE_CHAIN
        else:
            marker = sat_sub_u8(g, 40)
            op = OP_DILATE_REC if to_stab[i] else OP_DILATE_CHAIN
        dtype = "u8" if i < n_items // 2 else "f32"
        if dtype == "f32":
            marker = (marker.astype(np.float32) / np.float32(255.0)).astype(np.float32)
            g = (g.astype(np.float32) / np.float32(255.0)).astype(np.float32)
        items.append({"op": op, "dtype": dtype, "conn": 8 if conn8[i] else 4,
                      "steps": -1 if to_stab[i] else int(steps[i]),
                      "marker": marker, "mask": g})
    return items


def workload4(B: int = 32, H: int = 512, W: int = 512, dtype=np.float32, seed: int = SEED_BASE + 4):
    """Differentiable workload: mask = 3x3 box mean of U[0,1) + N(0,1e-4), marker = mask - U[0,0.2].

    Also returns the upstream gradient grad_out ~ N(0, 1). Arrays are (B, H, W).
    """
    n = B * H * W
    u = uniform01(seed, 41, n).reshape(B, H, W)
    mask = np.stack([box_mean_f64(u[b], 1) for b in range(B)])
    mask = mask + 1e-4 * normal(seed, 42, n).reshape(B, H, W)
    marker = mask - 0.2 * uniform01(seed, 43, n).reshape(B, H, W)
    grad = normal(seed, 44, n).reshape(B, H, W)
    return {"mask": mask.astype(dtype), "marker": marker.astype(dtype), "grad_out": grad.astype(dtype)}
