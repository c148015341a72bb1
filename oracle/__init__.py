"""CPU oracle for geodesic 3x3 chains -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package. The product path (``paper_1911_13074_gb300``)
never imports it and has no CPU fallback.

The arithmetic lives in ``oracle.c`` (plain C loops written from the paper's
definitions: Section 2, Eq. 1-5 for windows, steps, chains and
reconstruction, Eq. 6-12 for the geodesic operators, Eq. 13-15 and
Algorithm 6 for the quasi-distance transform, Eq. 16-20 for openings,
closings, granulometry and ASF, plus the reverse mode of the chain; see the
header of that file). This module builds it with gcc into
``oracle/_build/liboracle.so`` and converts numpy arrays to and from float64
around each call. uint8 and float32 values convert to float64 exactly and
the forward operators only select, so the results convert back exactly.

Parity pins: every function is checked against independent results in
``tests/test_oracle_pins.py`` (brute-force windows, scipy's max/min filters,
a van Herk / Gil-Werman running extreme, threshold decomposition with
breadth-first search, a widest-path search for reconstruction, finite
differences and a source-identity closed form for the backward pass),
``tests/test_oracle_ops_pins.py``, ``tests/test_oracle_qdt_pins.py`` and
``tests/test_oracle_gran_pins.py``; ``tests/test_oracle_mutants.py`` checks
that the pins catch planted mistakes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

DILATE, ERODE = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain -O2, no vector intrinsics)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_OMP_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_omp.so")
_omp_lib = None


def build_openmp(force: bool = False) -> str:
    """The same oracle.c compiled with -fopenmp: its step splits the rows of
    the image over OpenMP threads (OMP_NUM_THREADS), the arithmetic unchanged.
    Used only for the benchmark's all-core CPU baseline."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_OMP_LIB_PATH)
            and os.path.getmtime(_OMP_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _OMP_LIB_PATH
    tmp = _OMP_LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC])
    os.replace(tmp, _OMP_LIB_PATH)
    return _OMP_LIB_PATH


def chain_openmp(f, m, steps, conn=8, op="dilate"):
    """oracle.chain through the OpenMP build (one chain on OMP_NUM_THREADS threads)."""
    global _omp_lib
    with _lock:
        if _omp_lib is None:
            lib = ctypes.CDLL(build_openmp())
            P, L, I = ctypes.c_void_p, ctypes.c_long, ctypes.c_int
            lib.oracle_chain.argtypes = [P, P, P, L, L, I, I, L]
            lib.oracle_chain.restype = I
            _omp_lib = lib
    f64 = _f64(f)
    m64 = None if m is None else _f64(m)
    out = np.empty_like(f64)
    H, W = f64.shape
    if _omp_lib.oracle_chain(_ptr(f64), _ptr(m64), _ptr(out), H, W, conn, _opcode(op), int(steps)) != 0:
        raise MemoryError("oracle_chain failed")
    return _back(out, np.asarray(f))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            L = ctypes.c_long
            I = ctypes.c_int
            lib.oracle_step.argtypes = [P, P, P, L, L, I, I]
            lib.oracle_step.restype = None
            lib.oracle_chain.argtypes = [P, P, P, L, L, I, I, L]
            lib.oracle_chain.restype = I
            lib.oracle_reconstruct.argtypes = [P, P, P, L, L, I, I, L]
            lib.oracle_reconstruct.restype = L
            lib.oracle_window.argtypes = [P, P, L, L, L, I]
            lib.oracle_window.restype = I
            lib.oracle_chain_backward.argtypes = [P, P, P, P, P, L, L, I, I, L]
            lib.oracle_chain_backward.restype = I
            D = ctypes.c_double
            for name in ("oracle_hmax", "oracle_dome"):
                getattr(lib, name).argtypes = [P, P, L, L, I, D, D, I]
                getattr(lib, name).restype = L
            lib.oracle_hfill.argtypes = [P, P, L, L, I]
            lib.oracle_hfill.restype = L
            lib.oracle_raobj.argtypes = [P, P, L, L, I, I]
            lib.oracle_raobj.restype = L
            lib.oracle_open_rec.argtypes = [P, P, L, L, I, L]
            lib.oracle_open_rec.restype = L
            lib.oracle_qdt_residual.argtypes = [P, P, P, L, L, I, L]
            lib.oracle_qdt_residual.restype = I
            lib.oracle_qdt_lipschitz.argtypes = [P, P, L, L, I, L]
            lib.oracle_qdt_lipschitz.restype = L
            for name in ("oracle_opening", "oracle_closing", "oracle_asf"):
                getattr(lib, name).argtypes = [P, P, L, L, L]
                getattr(lib, name).restype = I
            lib.oracle_granulometry.argtypes = [P, L, L, L, P]
            lib.oracle_granulometry.restype = I
            _lib = lib
    return _lib


def use_library(path):
    """Load the oracle from another build of oracle.c (used by the mutation
    tests, which compile deliberately broken copies). Returns the previous
    library handle so the caller can restore it with ``restore_library``."""
    global _lib
    prev = _load()
    lib = ctypes.CDLL(path)
    for name in ("oracle_step", "oracle_chain", "oracle_reconstruct", "oracle_window",
                 "oracle_chain_backward", "oracle_hmax", "oracle_dome", "oracle_hfill", "oracle_raobj",
                 "oracle_open_rec", "oracle_qdt_residual", "oracle_qdt_lipschitz", "oracle_opening",
                 "oracle_closing", "oracle_granulometry", "oracle_asf"):
        fn, ref = getattr(lib, name), getattr(prev, name)
        fn.argtypes, fn.restype = ref.argtypes, ref.restype
    with _lock:
        _lib = lib
    return prev


def restore_library(prev):
    global _lib
    with _lock:
        _lib = prev


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _back(out64, like):
    if like.dtype == np.float64:
        return out64
    return out64.astype(like.dtype)


def _opcode(op):
    return {"dilate": DILATE, "erode": ERODE, DILATE: DILATE, ERODE: ERODE}[op]


def step(f, m, conn=8, op="dilate"):
    """One elementary geodesic step (Eq. 3 / its dual); m=None: plain 3x3 step."""
    lib = _load()
    f64 = _f64(f)
    m64 = None if m is None else _f64(m)
    out = np.empty_like(f64)
    H, W = f64.shape
    lib.oracle_step(_ptr(f64), _ptr(m64), _ptr(out), H, W, conn, _opcode(op))
    return _back(out, np.asarray(f))


def chain(f, m, steps, conn=8, op="dilate"):
    """Geodesic chain of `steps` elementary steps (Eq. 4); m=None: unmasked."""
    lib = _load()
    f64 = _f64(f)
    m64 = None if m is None else _f64(m)
    out = np.empty_like(f64)
    H, W = f64.shape
    rc = lib.oracle_chain(_ptr(f64), _ptr(m64), _ptr(out), H, W, conn, _opcode(op), int(steps))
    if rc != 0:
        raise MemoryError("oracle_chain failed")
    return _back(out, np.asarray(f))


def reconstruct(f, m, conn=8, op="dilate", max_steps=None):
    """Reconstruction by dilation / erosion (Eq. 5). Returns (out, changing_steps)."""
    lib = _load()
    f64 = _f64(f)
    m64 = _f64(m)
    out = np.empty_like(f64)
    H, W = f64.shape
    if max_steps is None:
        max_steps = H * W + 1
    n = lib.oracle_reconstruct(_ptr(f64), _ptr(m64), _ptr(out), H, W, conn, _opcode(op), int(max_steps))
    if n == -2:
        raise MemoryError("oracle_reconstruct failed")
    return _back(out, np.asarray(f)), int(n)


def window(f, half_size, op="dilate"):
    """Erosion / dilation by the clipped (2s+1)^2 square (Eq. 1-2)."""
    lib = _load()
    f64 = _f64(f)
    out = np.empty_like(f64)
    H, W = f64.shape
    rc = lib.oracle_window(_ptr(f64), _ptr(out), H, W, int(half_size), _opcode(op))
    if rc != 0:
        raise MemoryError("oracle_window failed")
    return _back(out, np.asarray(f))


def chain_backward(f, m, grad_out, steps, conn=8, op="dilate"):
    """Reverse mode of the masked chain. Returns (grad_marker, grad_mask) in float64."""
    lib = _load()
    f64, m64, g64 = _f64(f), _f64(m), _f64(grad_out)
    gmk = np.empty_like(f64)
    gms = np.empty_like(f64)
    H, W = f64.shape
    rc = lib.oracle_chain_backward(_ptr(f64), _ptr(m64), _ptr(g64), _ptr(gmk), _ptr(gms),
                                   H, W, conn, _opcode(op), int(steps))
    if rc != 0:
        raise MemoryError("oracle_chain_backward failed")
    return gmk, gms


# ---------------------------------------------------------------------------
# geodesic operators (Section 2, Eq. 6-12)
# ---------------------------------------------------------------------------

def _op_call(name, f, *args):
    lib = _load()
    f64 = _f64(f)
    out = np.empty_like(f64)
    H, W = f64.shape
    r = getattr(lib, name)(_ptr(f64), _ptr(out), H, W, *args)
    if r == -2:
        raise MemoryError(name)
    return _back(out, np.asarray(f))


def _lo(f):
    return 0.0 if np.asarray(f).dtype == np.uint8 else -np.inf


def _f32(f):
    return 1 if np.asarray(f).dtype == np.float32 else 0


def _h(f, h):
    # uint8 images take an integral h (rounded down); float images take h as
    # given, rounded to float32 for float32 images inside the oracle
    return float(np.floor(h)) if np.asarray(f).dtype == np.uint8 else float(h)


def hmax(f, h, conn=8):
    """HMAX_h(f) = delta_rec^f(f - h) (Eq. 6); the u8 marker saturates at 0."""
    return _op_call("oracle_hmax", f, conn, _h(f, h), _lo(f), _f32(f))


def dome(f, h, conn=8):
    """DOME_h(f) = f - HMAX_h(f) (Eq. 7)."""
    return _op_call("oracle_dome", f, conn, _h(f, h), _lo(f), _f32(f))


def hfill(f, conn=8):
    """HFILL(f) = eps_rec^f(m_HFILL(f)) (Eq. 8-9)."""
    return _op_call("oracle_hfill", f, conn)


def raobj(f, conn=8):
    """RAOBJ(f) = f - delta_rec^f(m_RAOBJ(f)) (Eq. 10-11)."""
    return _op_call("oracle_raobj", f, conn, _f32(f))


def open_rec(f, s, conn=8):
    """gamma_rec^s(f) = delta_rec^f(eps_s(f)) (Eq. 12)."""
    return _op_call("oracle_open_rec", f, conn, int(s))


# ---------------------------------------------------------------------------
# quasi-distance transform (Section 2, Eq. 13-15; Algorithm 6)
# ---------------------------------------------------------------------------

def qdt_steps(H, W, conn=8):
    """Number of eps_1 erosions after which eps_j(f) is constant on an H x W
    image: the clipped square of half size max(H, W) - 1 (the cross of radius
    H + W - 2) covers the whole image from every pixel."""
    if H == 0 or W == 0:
        return 0
    return max(H, W) - 1 if conn == 8 else H + W - 2


def qdt_residual(f, conn=8, steps=None):
    """d(f) of Eq. 13 as Algorithm 6 computes it. Returns (r, d): the largest
    residual eps_{j-1}(f) - eps_j(f) over the erosions j = 1..steps (f's dtype)
    and the first j that attains it (int32; 0 where no erosion lowers the
    pixel)."""
    lib = _load()
    f64 = _f64(f)
    H, W = f64.shape
    if steps is None:
        steps = qdt_steps(H, W, conn)
    r = np.empty_like(f64)
    d = np.empty_like(f64)
    if lib.oracle_qdt_residual(_ptr(f64), _ptr(r), _ptr(d), H, W, conn, int(steps)) != 0:
        raise MemoryError("oracle_qdt_residual failed")
    return _back(r, np.asarray(f)), d.astype(np.int32)


def qdt_lipschitz(g, conn=8, max_steps=None):
    """The limit of eta (Eq. 14-15) applied to g. Returns (out int32, changing
    steps)."""
    lib = _load()
    g64 = _f64(g)
    H, W = g64.shape
    out = np.empty_like(g64)
    if max_steps is None:
        max_steps = H * W + 1
    n = lib.oracle_qdt_lipschitz(_ptr(g64), _ptr(out), H, W, conn, int(max_steps))
    if n == -2:
        raise MemoryError("oracle_qdt_lipschitz failed")
    return out.astype(np.int32), int(n)


def qdt(f, conn=8):
    """Quasi-distance transform: (r, d, d_L1) with d_L1 the eta limit of d."""
    r, d = qdt_residual(f, conn)
    dl1, _ = qdt_lipschitz(d, conn)
    return r, d, dl1


# ---------------------------------------------------------------------------
# granulometry and alternating sequential filters (Section 2, Eq. 16-20)
# ---------------------------------------------------------------------------

def _win_call(name, f, s):
    lib = _load()
    f64 = _f64(f)
    out = np.empty_like(f64)
    H, W = f64.shape
    if getattr(lib, name)(_ptr(f64), _ptr(out), H, W, int(s)) != 0:
        raise MemoryError(name)
    return _back(out, np.asarray(f))


def opening(f, s):
    """gamma_s(f) = delta_s(eps_s(f)) as 2s elementary 3x3 steps (Eq. 16)."""
    return _win_call("oracle_opening", f, s)


def closing(f, s):
    """phi_s(f) = eps_s(delta_s(f)) (Eq. 19)."""
    return _win_call("oracle_closing", f, s)


def asf(f, s):
    """ASF_s(f) = phi_s gamma_s ... phi_1 gamma_1 (f) (Eq. 20)."""
    return _win_call("oracle_asf", f, s)


def granulometry(f, smax):
    """(G, PS): G_s = sum of gamma_s(f) for s = 0..smax (Eq. 17) and the
    pattern spectrum PS_s = G_s - G_{s+1} for s = 0..smax-1 (Eq. 18)."""
    lib = _load()
    f64 = _f64(f)
    H, W = f64.shape
    G = np.empty(int(smax) + 1, np.float64)
    if lib.oracle_granulometry(_ptr(f64), H, W, int(smax), _ptr(G)) != 0:
        raise MemoryError("oracle_granulometry")
    return G, G[:-1] - G[1:]
