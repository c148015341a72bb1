"""Pins for the CPU oracle: each oracle function checked against something other than itself.

The paper prints no worked numeric example, so the pins are independent
computations of the same mathematical objects:

* windows (Section 2, Eq. 1-2): a 2-D brute-force window, scipy.ndimage's
  max/min filters, and the decomposition claim of Section 3.1 (s chained 3x3
  steps give the (2s+1)^2 window);
* masked chains (Eq. 3-4): threshold decomposition -- flat operators commute
  with thresholding, so each level set of the chain is a breadth-first
  search inside the mask's level set;
* reconstruction (Eq. 5): a widest-path (max-min) Dijkstra search, connected
  component labelling per level, the fixed-point property and idempotence;
* the backward pass (not in the paper): central finite differences and the
  source-identity closed form on tie-free float64 inputs.

A plausible slip in the oracle (a dropped neighbour, a wrong clamp direction,
a transposed index, an off-by-one in the border clipping or the step count)
fails at least one of these.
"""
import heapq
from collections import deque

import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth

RNG = np.random.default_rng(12345)


def shape_offsets(conn):
    if conn == 8:
        return [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    return [(-1, 0), (0, -1), (0, 0), (0, 1), (1, 0)]


def brute_window(f, s, op):
    H, W = f.shape
    out = np.empty_like(f)
    for y in range(H):
        for x in range(W):
            blk = f[max(0, y - s):y + s + 1, max(0, x - s):x + s + 1]
            out[y, x] = blk.max() if op == "dilate" else blk.min()
    return out


def brute_diamond(f, r, op):
    H, W = f.shape
    out = np.empty_like(f)
    for y in range(H):
        for x in range(W):
            vals = [f[qy, qx] for qy in range(max(0, y - r), min(H, y + r + 1))
                    for qx in range(max(0, x - r), min(W, x + r + 1))
                    if abs(qy - y) + abs(qx - x) <= r]
            out[y, x] = max(vals) if op == "dilate" else min(vals)
    return out


def geodesic_bfs(src, allowed, conn):
    """Multi-source BFS distance: sources at 0, expansion only into `allowed`."""
    H, W = src.shape
    dist = np.full((H, W), np.iinfo(np.int64).max, np.int64)
    dq = deque()
    for y, x in zip(*np.nonzero(src)):
        dist[y, x] = 0
        dq.append((y, x))
    offs = [o for o in shape_offsets(conn) if o != (0, 0)]
    while dq:
        y, x = dq.popleft()
        d = dist[y, x] + 1
        for dy, dx in offs:
            qy, qx = y + dy, x + dx
            if 0 <= qy < H and 0 <= qx < W and allowed[qy, qx] and dist[qy, qx] > d:
                dist[qy, qx] = d
                dq.append((qy, qx))
    return dist


def chain_by_thresholds(f, m, steps, conn, op):
    """Masked chain via threshold decomposition + BFS (independent of the step loop)."""
    levels = np.unique(np.concatenate([f.ravel(), m.ravel()]))
    if op == "dilate":
        out = np.full(f.shape, -np.inf)
        for t in levels:
            F, M = f >= t, m >= t
            if steps == 0:
                X = F
            else:
                X = M & (geodesic_bfs(F, M, conn) <= steps)
            out[X] = np.maximum(out[X], t)
        # every pixel lies in X at the lowest level present: out is finite
    else:
        out = np.full(f.shape, np.inf)
        for t in levels:
            F, M = f <= t, m <= t
            X = F if steps == 0 else (M & (geodesic_bfs(F, M, conn) <= steps))
            out[X] = np.minimum(out[X], t)
    return out


def widest_path_reconstruct(f, m, conn, op):
    """Reconstruction as a max-min path problem solved by Dijkstra.

    rec(p) = max over walks r0 -> r1 -> ... -> rn = p (n >= 1, neighbours in the
    connectivity, staying in place allowed) of min(f(r0), m(r1), ..., m(rn)).
    Erosion is the same problem on negated values.
    """
    if op == "erode":
        return -widest_path_reconstruct(-f, -m, conn, "dilate")
    H, W = f.shape
    offs = shape_offsets(conn)
    best = np.full((H, W), -np.inf)
    for y in range(H):
        for x in range(W):
            for dy, dx in offs:
                qy, qx = y + dy, x + dx
                if 0 <= qy < H and 0 <= qx < W:
                    best[y, x] = max(best[y, x], min(f[qy, qx], m[y, x]))
    heap = [(-best[y, x], y, x) for y in range(H) for x in range(W)]
    heapq.heapify(heap)
    done = np.zeros((H, W), bool)
    while heap:
        nb, y, x = heapq.heappop(heap)
        if done[y, x]:
            continue
        done[y, x] = True
        b = -nb
        for dy, dx in offs:
            qy, qx = y + dy, x + dx
            if 0 <= qy < H and 0 <= qx < W and not done[qy, qx]:
                c = min(b, m[qy, qx])
                if c > best[qy, qx]:
                    best[qy, qx] = c
                    heapq.heappush(heap, (-c, qy, qx))
    return best


def rand_img(H, W, kind):
    if kind == "u8":
        return RNG.integers(0, 256, (H, W)).astype(np.uint8)
    if kind == "u8few":
        return (RNG.integers(0, 6, (H, W)) * 40).astype(np.uint8)
    if kind == "f32":
        return RNG.random((H, W)).astype(np.float32)
    return RNG.random((H, W))


# ---------------------------------------------------------------------------
# Windows and unmasked chains (Eq. 1-2, Section 3.1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_window_matches_bruteforce_and_chain_on_tiny_images(op):
    for H in range(1, 10):
        for W in range(1, 10):
            f = rand_img(H, W, "u8")
            for s in range(0, 6):
                ref = brute_window(f, s, op)
                np.testing.assert_array_equal(oracle.window(f, s, op), ref)
                np.testing.assert_array_equal(oracle.chain(f, None, s, conn=8, op=op), ref)


@pytest.mark.parametrize("kind", ["u8", "f32", "f64"])
@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_window_matches_scipy_filters(kind, op):
    f = rand_img(37, 53, kind)
    for s in (1, 2, 7, 13, 30):
        filt = ndimage.maximum_filter if op == "dilate" else ndimage.minimum_filter
        ref = filt(f, size=2 * s + 1, mode="nearest")
        np.testing.assert_array_equal(oracle.window(f, s, op), ref)
        np.testing.assert_array_equal(oracle.chain(f, None, s, conn=8, op=op), ref)


@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_four_connected_chain_is_clipped_diamond(op):
    for H, W in [(1, 1), (1, 7), (6, 1), (5, 8), (11, 9)]:
        f = rand_img(H, W, "u8")
        for r in range(0, 7):
            np.testing.assert_array_equal(oracle.chain(f, None, r, conn=4, op=op),
                                          brute_diamond(f, r, op))
    f = rand_img(40, 31, "f64")
    for r in (3, 9):
        fp = ndimage.generate_binary_structure(2, 1)
        fp = ndimage.iterate_structure(fp, r)
        g = ndimage.grey_dilation if op == "dilate" else ndimage.grey_erosion
        np.testing.assert_array_equal(oracle.chain(f, None, r, conn=4, op=op),
                                      g(f, footprint=fp, mode="nearest"))


def van_herk_1d(x, s, op, axis):
    """Running extreme of window 2s+1 along `axis` by the van Herk / Gil-Werman
    method: pad with the identity, cut into blocks of the window length, take
    the prefix extreme g and the suffix extreme h inside every block; the
    window starting at i is then ext(h[i], g[i + 2s])."""
    ext = np.maximum if op == "dilate" else np.minimum
    ident = -np.inf if op == "dilate" else np.inf
    x = np.moveaxis(np.asarray(x, np.float64), axis, -1)
    n, w = x.shape[-1], 2 * s + 1
    nb = -(-(n + 2 * s) // w)
    xp = np.full(x.shape[:-1] + (nb * w,), ident)
    xp[..., s:s + n] = x
    blocks = xp.reshape(x.shape[:-1] + (nb, w))
    g = ext.accumulate(blocks, axis=-1).reshape(xp.shape)
    h = ext.accumulate(blocks[..., ::-1], axis=-1)[..., ::-1].reshape(xp.shape)
    i = np.arange(n)
    return np.moveaxis(ext(h[..., i], g[..., i + w - 1]), -1, axis)


@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_window_matches_van_herk_at_full_size(op):
    """The 1024x1024 workload-1 windows (s = 13 and 91) against a separable
    van Herk / Gil-Werman running extreme, rows then columns."""
    g = synth.workload1_u8()["mask"]
    for s in (13, 91):
        ref = van_herk_1d(van_herk_1d(g, s, op, 1), s, op, 0)
        np.testing.assert_array_equal(oracle.window(g, s, op).astype(np.float64), ref)


def test_window_on_workload_image():
    g = synth.workload0(96, 80)["mask"]
    for s in (13, 40):
        for op, filt in (("dilate", ndimage.maximum_filter), ("erode", ndimage.minimum_filter)):
            np.testing.assert_array_equal(oracle.window(g, s, op),
                                          filt(g, size=2 * s + 1, mode="nearest"))


# ---------------------------------------------------------------------------
# Masked chains (Eq. 3-4)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("op", ["dilate", "erode"])
@pytest.mark.parametrize("kind", ["u8few", "f64"])
def test_masked_chain_threshold_decomposition(conn, op, kind):
    for H, W in [(1, 1), (1, 9), (7, 1), (9, 13), (16, 12)]:
        f = rand_img(H, W, kind)
        m = rand_img(H, W, kind)
        for steps in (0, 1, 2, 3, 5, 17):
            got = oracle.chain(f, m, steps, conn=conn, op=op)
            ref = chain_by_thresholds(f.astype(np.float64), m.astype(np.float64), steps, conn, op)
            np.testing.assert_array_equal(got.astype(np.float64), ref)


@pytest.mark.parametrize("conn", [4, 8])
def test_masked_chain_threshold_decomposition_workload(conn):
    w = synth.workload0(40, 36)
    f, m = w["marker"], w["mask"]
    # quantise to 12 levels so the per-level BFS stays cheap; still a valid pair
    fq = (f // 22) * 22
    mq = (m // 22) * 22
    for steps in (4, 25):
        got = oracle.chain(fq, mq, steps, conn=conn)
        ref = chain_by_thresholds(fq.astype(np.float64), mq.astype(np.float64), steps, conn, "dilate")
        np.testing.assert_array_equal(got.astype(np.float64), ref)


def test_masked_chain_invariants():
    w = synth.workload0(64, 64)
    f, m = w["marker"], w["mask"]
    prev = f
    for steps in (1, 2, 5, 20, 64):
        out = oracle.chain(f, m, steps, conn=8)
        assert np.all(f <= out) and np.all(out <= m)
        assert np.all(prev <= out)  # monotone in the number of steps
        prev = out
    # monotone in the marker and in the mask
    f2 = np.minimum(f.astype(np.int64) + 7, m).astype(np.uint8)
    assert np.all(oracle.chain(f, m, 10) <= oracle.chain(f2, m, 10))
    m2 = np.minimum(m.astype(np.int64) + 9, 255).astype(np.uint8)
    assert np.all(oracle.chain(f, m, 10) <= oracle.chain(f, m2, 10))


@pytest.mark.parametrize("conn", [4, 8])
def test_erosion_dilation_duality(conn):
    w = synth.workload1_u8(48, 40)
    f, m = w["marker_erode"], w["mask"]
    ero = oracle.chain(f, m, 9, conn=conn, op="erode")
    dil = oracle.chain(255 - f, 255 - m, 9, conn=conn, op="dilate")
    np.testing.assert_array_equal(ero, 255 - dil)
    wf = synth.workload1_f64(24, 30)
    ero = oracle.chain(wf["marker_erode"], wf["mask"], 7, conn=conn, op="erode")
    dil = oracle.chain(-wf["marker_erode"], -wf["mask"], 7, conn=conn, op="dilate")
    np.testing.assert_array_equal(ero, -dil)


# ---------------------------------------------------------------------------
# Reconstruction (Eq. 5)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("op", ["dilate", "erode"])
@pytest.mark.parametrize("kind", ["u8", "f32", "f64"])
def test_reconstruct_is_widest_path(conn, op, kind):
    for H, W in [(1, 1), (1, 12), (10, 1), (13, 17), (30, 25)]:
        f = rand_img(H, W, kind)
        m = rand_img(H, W, kind)
        rec, n = oracle.reconstruct(f, m, conn=conn, op=op)
        ref = widest_path_reconstruct(f.astype(np.float64), m.astype(np.float64), conn, op)
        np.testing.assert_array_equal(rec.astype(np.float64), ref)
        # the chain reaches the same image after exactly n changing steps
        np.testing.assert_array_equal(oracle.chain(f, m, n, conn=conn, op=op), rec)
        if n > 0:
            assert not np.array_equal(oracle.chain(f, m, n - 1, conn=conn, op=op), rec)


@pytest.mark.parametrize("conn", [4, 8])
def test_reconstruct_workload0_fixed_point_and_components(conn):
    w = synth.workload0(128, 112)
    f, m = w["marker"], w["mask"]
    rec, n = oracle.reconstruct(f, m, conn=conn)
    assert n > 0
    np.testing.assert_array_equal(oracle.step(rec, m, conn=conn), rec)          # fixed point
    np.testing.assert_array_equal(oracle.reconstruct(rec, m, conn=conn)[0], rec)  # idempotent
    assert np.all(f <= rec) and np.all(rec <= m)
    # level sets: {rec >= t} = union of the connected components of {m >= t}
    # that meet delta_1({f >= t})
    st = ndimage.generate_binary_structure(2, 2 if conn == 8 else 1)
    for t in range(1, 256, 5):
        M = m >= t
        seed_set = ndimage.binary_dilation(f >= t, structure=st) & M
        lab, _ = ndimage.label(M, structure=st)
        keep = np.unique(lab[seed_set])
        keep = keep[keep > 0]
        np.testing.assert_array_equal(rec >= t, np.isin(lab, keep))


def test_reconstruct_reports_not_converged():
    w = synth.workload0(32, 32)
    rec, n = oracle.reconstruct(w["marker"], w["mask"], max_steps=2)
    assert n == -1


# ---------------------------------------------------------------------------
# Backward pass (reverse mode of Eq. 4)
# ---------------------------------------------------------------------------

def tie_free_pair(H, W, seed):
    r = np.random.default_rng(seed)
    vals = r.permutation(2 * H * W).astype(np.float64) / (2 * H * W) + 0.25 / (2 * H * W)
    m = vals[:H * W].reshape(H, W).copy()
    f = vals[H * W:].reshape(H, W).copy()
    # a valid dilation pair keeps many mask selections and many marker paths
    lo = np.minimum(f, m)
    hi = np.maximum(f, m)
    return lo, hi


def fd_gradient(f, m, g, steps, conn, op, wrt, h):
    """Central differences, summed per output pixel (each difference is exact)."""
    x = (f if wrt == "marker" else m)
    grad = np.zeros_like(x)
    for i in range(x.size):
        xp = x.copy()
        xm = x.copy()
        xp.flat[i] += h
        xm.flat[i] -= h
        if wrt == "marker":
            op_ = oracle.chain(xp, m, steps, conn=conn, op=op)
            om_ = oracle.chain(xm, m, steps, conn=conn, op=op)
        else:
            op_ = oracle.chain(f, xp, steps, conn=conn, op=op)
            om_ = oracle.chain(f, xm, steps, conn=conn, op=op)
        d = (op_ - om_) / (2 * h)  # entries are exactly 0 or 1
        assert np.all((d == 0) | (d == 1))
        grad.flat[i] = float(np.sum(g[d == 1]))
    return grad


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_backward_matches_finite_differences(conn, op):
    H, W, steps = 7, 9, 5
    lo, hi = tie_free_pair(H, W, 7 + conn)
    f, m = (lo, hi) if op == "dilate" else (hi, lo)
    g = np.random.default_rng(3).standard_normal((H, W))
    gmk, gms = oracle.chain_backward(f, m, g, steps, conn=conn, op=op)
    h = 2.0 ** -30  # far below the smallest value gap (1 / 126)
    np.testing.assert_allclose(gmk, fd_gradient(f, m, g, steps, conn, op, "marker", h), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(gms, fd_gradient(f, m, g, steps, conn, op, "mask", h), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_backward_source_identity(conn, op):
    """With all input values distinct, each output is a copy of exactly one input element."""
    H, W, steps = 23, 19, 11
    lo, hi = tie_free_pair(H, W, 99 + conn)
    f, m = (lo, hi) if op == "dilate" else (hi, lo)
    # also break validity in a few pixels: the first step then clamps to the mask
    f = f.copy()
    f[3, 4], m[3, 4] = m[3, 4], f[3, 4]
    g = np.random.default_rng(5).standard_normal((H, W))
    out = oracle.chain(f, m, steps, conn=conn, op=op)
    where = {}
    for i, v in enumerate(f.ravel()):
        where[v] = ("marker", i)
    for i, v in enumerate(m.ravel()):
        where[v] = ("mask", i)
    exp_mk = np.zeros(H * W)
    exp_ms = np.zeros(H * W)
    for p, v in enumerate(out.ravel()):
        kind, i = where[v]
        (exp_mk if kind == "marker" else exp_ms)[i] += g.ravel()[p]
    gmk, gms = oracle.chain_backward(f, m, g, steps, conn=conn, op=op)
    np.testing.assert_allclose(gmk.ravel(), exp_mk, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(gms.ravel(), exp_ms, rtol=1e-12, atol=1e-12)


def test_backward_tie_rule_lowest_index_and_marker_on_mask_tie():
    """Plateau inputs: a tie must route to the lowest neighbour index k, and a
    mask equal to the neighbourhood maximum must keep the marker branch."""
    f = np.array([[1.0, 1.0, 0.0],
                  [0.0, 0.5, 0.0],
                  [0.0, 0.0, 1.0]])
    m = np.full((3, 3), 1.0)
    g = np.zeros((3, 3))
    g[1, 1] = 1.0
    gmk, gms = oracle.chain_backward(f, m, g, 1, conn=8)
    # centre (1,1): maxima 1.0 at k=0 (0,0), k=1 (0,1), k=8 (2,2) -> k=0 wins; m == v keeps marker
    exp = np.zeros((3, 3))
    exp[0, 0] = 1.0
    np.testing.assert_array_equal(gmk, exp)
    np.testing.assert_array_equal(gms, np.zeros((3, 3)))
    # with m strictly below the maximum the gradient goes to the mask
    m2 = m.copy()
    m2[1, 1] = 0.75
    gmk, gms = oracle.chain_backward(f, m2, g, 1, conn=8)
    np.testing.assert_array_equal(gmk, np.zeros((3, 3)))
    assert gms[1, 1] == 1.0 and gms.sum() == 1.0
    # 4-connectivity ignores the diagonal (0,0): k=1 (0,1) wins
    gmk, _ = oracle.chain_backward(f, m, g, 1, conn=4)
    exp = np.zeros((3, 3))
    exp[0, 1] = 1.0
    np.testing.assert_array_equal(gmk, exp)


def test_empty_and_degenerate_images():
    e = np.zeros((0, 5), np.uint8)
    assert oracle.chain(e, e, 3).shape == (0, 5)
    assert oracle.window(e, 2).shape == (0, 5)
    one = np.array([[7]], np.uint8)
    assert oracle.chain(one, np.array([[9]], np.uint8), 100)[0, 0] == 7
    assert oracle.chain(np.array([[9]], np.uint8), np.array([[7]], np.uint8), 1)[0, 0] == 7
    assert oracle.window(one, 50)[0, 0] == 7


def test_backward_erosion_tie_rule():
    """Dual of the plateau case: lowest k among the minima; mask equal to the minimum keeps the marker."""
    f = np.array([[0.0, 0.0, 1.0],
                  [1.0, 0.5, 1.0],
                  [1.0, 1.0, 0.0]])
    m = np.zeros((3, 3))
    g = np.zeros((3, 3))
    g[1, 1] = 1.0
    gmk, gms = oracle.chain_backward(f, m, g, 1, conn=8, op="erode")
    exp = np.zeros((3, 3))
    exp[0, 0] = 1.0
    np.testing.assert_array_equal(gmk, exp)
    np.testing.assert_array_equal(gms, np.zeros((3, 3)))
