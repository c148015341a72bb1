// Reverse mode of the masked geodesic chain (Eq. 3-4) for float32 / float64.
//
// The paper has no backward pass; this library differentiates its chains
// with these rules. A step maps f_{t-1} to f_t with
//   f_t(p) = clamp(ext_{q in N(p)} f_{t-1}(q), m(p)),
// where ext is max (dilation) or min (erosion) over the clipped neighbourhood
// and clamp the opposite extreme with the mask. Each output value is a copy
// of one input value, so the Jacobian routes the upstream gradient g_t(p):
//   * to the mask at p when the mask is strictly beyond the neighbourhood
//     extreme (m(p) < v for dilation, m(p) > v for erosion);
//   * otherwise to f_{t-1}(p + d_k), k the lowest neighbour index
//     k = (dy+1)*3 + (dx+1) that attains the extreme.
// The chain rule is applied as a gather, so no atomics are needed and the
// result does not depend on scheduling:
//   g_{t-1}(q) = sum over k = 0..8, in increasing k, of g_t(q - d_k)
//                where pixel q - d_k is in the image and routed to k,
//   grad_mask(p) += g_t(p) where p routed to the mask, for t = N, ..., 1.
//
// Memory: the forward pass stores checkpoints f_{sC} every C steps
// (geo_chain_fwd_ckpt). The backward pass walks the segments from last to
// first. Per segment, the chain kernel recomputes the states at every 8th
// step from the checkpoint; then, per sub-segment of up to 8 steps (last
// first), one fused kernel per 64x64 tile (32x32 for float64) recomputes the
// forward in shared memory from the sub-segment start, keeping one routing
// byte per pixel and step (0..8 = neighbour, 9 = mask), and replays the
// steps in reverse there: the gradient and grad_mask touch global memory
// once per sub-segment instead of once per step.
#include <cstring>

#include "geo_common.cuh"

namespace geo {
namespace {

constexpr uint8_t kRouteMask = 9;

template <int CONN>
__device__ __forceinline__ bool in_shape(int k) {
  return CONN == 8 || k == 1 || k == 3 || k == 4 || k == 5 || k == 7;
}

// Launch shape of the small per-pixel kernels: a 32 x 8 block of a row
// band, blockIdx.z = image of the batch.
constexpr int kBX = 32, kBY = 8;

// ---------------------------------------------------------------------------
// fused segment kernel: forward recompute and reverse replay of up to SS
// steps for one TT x TT tile, all in shared memory
// ---------------------------------------------------------------------------

constexpr int kSegT = 32;                  // the CTA is kSegT x kSegT threads
constexpr int kSegThreads = kSegT * kSegT;

template <typename T, int TT, int SS>
struct SegGeom {
  static constexpr int RF = TT + 4 * SS;  // forward region side: the tile plus 2 SS
  static constexpr int RB = TT + 2 * SS;  // reverse region side: the tile plus SS
  static constexpr size_t f_bytes = sizeof(T) * RF * RF;
  static constexpr size_t code_bytes = ((size_t)SS * RB * RB + 15) / 16 * 16;
  static constexpr size_t g_bytes = sizeof(T) * RB * RB;
  static constexpr size_t smem = 3 * f_bytes + code_bytes + 2 * g_bytes;
};

// One forward cell: neighbourhood extreme (lowest index on ties), mask branch.
// `checked`: clip the neighbourhood to the image (tiles near the border).
template <typename T, int OP, int CONN, int RF, bool checked>
__device__ __forceinline__ void seg_cell(const T *cur, const T *ms, int r, int c, int y, int x, int H, int W, T &out,
                                         uint8_t &code) {
  T best = T(0);
  int bk = -1;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    if (!in_shape<CONN>(k)) continue;
    const int dy = k / 3 - 1, dx = k % 3 - 1;
    if (checked && (y + dy < 0 || y + dy >= H || x + dx < 0 || x + dx >= W)) continue;
    const T v = cur[(r + dy) * RF + (c + dx)];
    if (bk < 0 || (OP == DILATE ? (v > best) : (v < best))) {
      best = v;
      bk = k;
    }
  }
  const T mv = ms[r * RF + c];
  const bool to_mask = (OP == DILATE) ? (mv < best) : (mv > best);
  out = to_mask ? mv : best;
  code = to_mask ? kRouteMask : (uint8_t)bk;
}

// f0: the state at the segment start, packed (row stride W). S <= SS steps
// t0+1 .. t0+S are recomputed; then g at t0+S (g_in) is carried back to t0
// (g_out) and grad_mask gathers the mask-routed gradients of those steps in
// decreasing step order (written, not accumulated, when `first`).
template <typename T, int OP, int CONN, int TT, int SS>
__global__ void __launch_bounds__(kSegThreads) seg_backward(const T *__restrict__ f0, const T *__restrict__ mask,
                                                            int64_t mpitch, const T *__restrict__ g_in,
                                                            int64_t gi_pitch, T *__restrict__ g_out, int64_t go_pitch,
                                                            T *__restrict__ gmask, int64_t gm_pitch, int H, int W,
                                                            int S, int first) {
  using G = SegGeom<T, TT, SS>;
  constexpr int RF = G::RF, RB = G::RB;
  extern __shared__ __align__(16) char smem[];
  T *fa = reinterpret_cast<T *>(smem);
  T *fb = reinterpret_cast<T *>(smem + G::f_bytes);
  T *ms = reinterpret_cast<T *>(smem + 2 * G::f_bytes);
  uint8_t *codes = reinterpret_cast<uint8_t *>(smem + 3 * G::f_bytes);
  T *ga = reinterpret_cast<T *>(smem + 3 * G::f_bytes + G::code_bytes);
  T *gb = reinterpret_cast<T *>(smem + 3 * G::f_bytes + G::code_bytes + G::g_bytes);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int b = blockIdx.z;
  const int ty0 = blockIdx.y * TT, tx0 = blockIdx.x * TT;
  const int fy0 = ty0 - 2 * SS, fx0 = tx0 - 2 * SS;  // forward region origin (global)
  const int by0 = ty0 - SS, bx0 = tx0 - SS;          // reverse region origin (global)
  // the whole forward region inside the image: no clipping needed anywhere
  const bool inner = fy0 >= 0 && fx0 >= 0 && fy0 + RF <= H && fx0 + RF <= W;
  const T *fimg = f0 + (size_t)b * H * W;
  const T *mimg = mask + (size_t)b * H * mpitch;
  // stage f0 and the mask on the forward region
  for (int r = ty; r < RF; r += kSegT) {
    const int y = fy0 + r;
    for (int c = tx; c < RF; c += kSegT) {
      const int x = fx0 + c;
      const bool in = y >= 0 && y < H && x >= 0 && x < W;
      fa[r * RF + c] = in ? fimg[(size_t)y * W + x] : T(0);
      ms[r * RF + c] = in ? mimg[(size_t)y * mpitch + x] : T(0);
    }
  }
  __syncthreads();
  // forward: step j computes the cells within 2SS - j of the tile and keeps
  // the routing codes of the cells within SS of it
  T *cur = fa, *nxt = fb;
  for (int j = 1; j <= S; ++j) {
    const int lo = j, hi = RF - j;  // rows / cols [lo, hi) of the forward region
    uint8_t *ct = codes + (size_t)(j - 1) * RB * RB;
    for (int r = lo + ty; r < hi; r += kSegT) {
      const int y = fy0 + r;
      for (int c = lo + tx; c < hi; c += kSegT) {
        const int x = fx0 + c;
        uint8_t code = 0xff;  // outside the image: matches no neighbour index
        T out = T(0);
        if (inner) {
          seg_cell<T, OP, CONN, RF, false>(cur, ms, r, c, y, x, H, W, out, code);
        } else if (y >= 0 && y < H && x >= 0 && x < W) {
          seg_cell<T, OP, CONN, RF, true>(cur, ms, r, c, y, x, H, W, out, code);
        }
        nxt[r * RF + c] = out;
        const int rb = r - SS, cb = c - SS;
        if (rb >= 0 && rb < RB && cb >= 0 && cb < RB) ct[rb * RB + cb] = code;
      }
    }
    __syncthreads();
    T *tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  // reverse: stage g at t0+S on the reverse region
  const T *gimg = g_in + (size_t)b * H * gi_pitch;
  for (int r = ty; r < RB; r += kSegT) {
    const int y = by0 + r;
    for (int c = tx; c < RB; c += kSegT) {
      const int x = bx0 + c;
      ga[r * RB + c] = (y >= 0 && y < H && x >= 0 && x < W) ? gimg[(size_t)y * gi_pitch + x] : T(0);
    }
  }
  // per thread: its fixed tile pixels' mask gradient, (ty + e * kSegT, tx + f * kSegT)
  constexpr int PT = (TT + kSegT - 1) / kSegT;
  T gmacc[PT][PT];
  T *gmimg = gmask + (size_t)b * H * gm_pitch;
#pragma unroll
  for (int e = 0; e < PT; ++e)
#pragma unroll
    for (int f = 0; f < PT; ++f) {
      const int r = ty + e * kSegT, c = tx + f * kSegT;
      const int y = ty0 + r, x = tx0 + c;
      gmacc[e][f] = (!first && r < TT && c < TT && y < H && x < W) ? gmimg[(size_t)y * gm_pitch + x] : T(0);
    }
  __syncthreads();
  T *gc = ga, *gn = gb;
  for (int j = S; j >= 1; --j) {
    const uint8_t *ct = codes + (size_t)(j - 1) * RB * RB;
    // grad_mask of the tile at step t0 + j, in decreasing step order
#pragma unroll
    for (int e = 0; e < PT; ++e)
#pragma unroll
      for (int f = 0; f < PT; ++f) {
        const int r = SS + ty + e * kSegT, c = SS + tx + f * kSegT;
        if (ty + e * kSegT < TT && tx + f * kSegT < TT && ct[r * RB + c] == kRouteMask) gmacc[e][f] += gc[r * RB + c];
      }
    // g at t0 + j - 1 on the cells within j - 1 of the tile
    const int lo = SS - (j - 1), hi = RB - lo;
    for (int r = lo + ty; r < hi; r += kSegT) {
      for (int c = lo + tx; c < hi; c += kSegT) {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          if (!in_shape<CONN>(k)) continue;
          const int pr = r - (k / 3 - 1), pc = c - (k % 3 - 1);
          if (ct[pr * RB + pc] == k) acc += gc[pr * RB + pc];
        }
        gn[r * RB + c] = acc;
      }
    }
    __syncthreads();
    T *tmp = gc;
    gc = gn;
    gn = tmp;
  }
  // write g at t0 and grad_mask for the tile
  T *goimg = g_out + (size_t)b * H * go_pitch;
#pragma unroll
  for (int e = 0; e < PT; ++e)
#pragma unroll
    for (int f = 0; f < PT; ++f) {
      const int r = ty + e * kSegT, c = tx + f * kSegT;
      const int y = ty0 + r, x = tx0 + c;
      if (r < TT && c < TT && y < H && x < W) {
        goimg[(size_t)y * go_pitch + x] = gc[(SS + r) * RB + SS + c];
        gmimg[(size_t)y * gm_pitch + x] = gmacc[e][f];
      }
    }
}

template <typename T>
__global__ void __launch_bounds__(kBX * kBY) zero_plane(T *__restrict__ p, int64_t pitch, int H, int W) {
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  if (x >= W || y >= H) return;
  p[(size_t)blockIdx.z * H * pitch + (size_t)y * pitch + x] = T(0);
}

// Sub-segment length of the fused kernel and its tile side per element type.
constexpr int kSeg = 8;
constexpr int kTileF32 = 64, kTileF64 = 32;

struct Layout {
  int64_t npx;    // batch * H * W
  int64_t nseg;   // checkpoints (segments of C steps)
  int64_t nsub;   // sub-segment starts kept per segment (C / kSeg, rounded up)
  size_t ckpt_b;  // bytes of one packed state (all images)
  size_t off_ckpt, off_state0, off_state1, off_sub, off_g0, off_g1, total;
};

Layout layout(int es, int64_t H, int64_t W, int64_t steps, int C, int batch) {
  Layout L{};
  L.npx = (int64_t)batch * H * W;
  L.nseg = steps > 0 ? (steps + C - 1) / C : 1;
  L.nsub = (C + kSeg - 1) / kSeg;
  L.ckpt_b = (size_t)L.npx * es;
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t st = up(L.ckpt_b);
  L.off_ckpt = 0;
  L.off_state0 = L.off_ckpt + st * (size_t)L.nseg;
  L.off_state1 = L.off_state0 + st;
  L.off_sub = L.off_state1 + st;
  L.off_g0 = L.off_sub + st * (size_t)L.nsub;
  L.off_g1 = L.off_g0 + st;
  L.total = L.off_g1 + st;
  return L;
}

dim3 step_grid(int64_t H, int64_t W, int batch) {
  return dim3((unsigned)((W + kBX - 1) / kBX), (unsigned)((H + kBY - 1) / kBY), (unsigned)batch);
}

template <typename T, int TT>
int launch_seg(int op, int conn, const T *f0, const T *mask, int64_t mpitch, const T *gin, int64_t gi_pitch, T *gout,
               int64_t go_pitch, T *gm, int64_t gm_pitch, int H, int W, int batch, int S, int first, cudaStream_t s) {
  using Gm = SegGeom<T, TT, kSeg>;
  const dim3 grid((unsigned)((W + TT - 1) / TT), (unsigned)((H + TT - 1) / TT), (unsigned)batch);
  void (*k)(const T *, const T *, int64_t, const T *, int64_t, T *, int64_t, T *, int64_t, int, int, int, int);
  if (op == DILATE) k = conn == 8 ? seg_backward<T, DILATE, 8, TT, kSeg> : seg_backward<T, DILATE, 4, TT, kSeg>;
  else k = conn == 8 ? seg_backward<T, ERODE, 8, TT, kSeg> : seg_backward<T, ERODE, 4, TT, kSeg>;
  if (cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::smem) !=
      cudaSuccess)
    return GEO_ERR_CUDA;
  k<<<grid, dim3(kSegT, kSegT), Gm::smem, s>>>(f0, mask, mpitch, gin, gi_pitch, gout, go_pitch, gm, gm_pitch, H, W, S,
                                                 first);
  return cudaGetLastError() == cudaSuccess ? GEO_OK : GEO_ERR_CUDA;
}

template <typename T>
int backward_impl(int dt, int op, int conn, const T *mask, const T *grad_out, T *grad_marker, T *grad_mask,
                  int64_t H64, int64_t W64, int64_t pitch, int64_t steps, int C, int batch, const char *ws,
                  cudaStream_t s) {
  constexpr int TT = sizeof(T) == 4 ? kTileF32 : kTileF64;
  const Layout Lw = layout((int)sizeof(T), H64, W64, steps, C, batch);
  const int H = (int)H64, W = (int)W64;
  const size_t st = (Lw.ckpt_b + 255) & ~(size_t)255;
  if (steps == 0) {
    zero_plane<T><<<dim3((unsigned)((W + kBX - 1) / kBX), (unsigned)((H + kBY - 1) / kBY), (unsigned)batch),
                    dim3(kBX, kBY), 0, s>>>(grad_mask, pitch, H, W);
    if (cudaMemcpy2DAsync(grad_marker, pitch * sizeof(T), grad_out, pitch * sizeof(T), W64 * sizeof(T),
                          H64 * (int64_t)batch, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return GEO_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? GEO_OK : GEO_ERR_CUDA;
  }
  char *w = const_cast<char *>(ws);
  // the sub-checkpoints come from the chain kernel, which takes one row
  // stride for all planes: keep a packed copy of the mask
  T *pmask = (T *)(w + Lw.off_state0);
  if (cudaMemcpy2DAsync(pmask, W64 * sizeof(T), mask, pitch * sizeof(T), W64 * sizeof(T), H64 * (int64_t)batch,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GEO_ERR_CUDA;
  T *gbuf[2] = {(T *)(w + Lw.off_g0), (T *)(w + Lw.off_g1)};
  const T *gcur = grad_out;  // the gradient being propagated and its row stride
  int64_t gcur_pitch = pitch;
  int gsel = 0;
  for (int64_t seg = Lw.nseg - 1; seg >= 0; --seg) {
    const int64_t t0 = seg * C;
    const int64_t t1 = (t0 + C < steps) ? t0 + C : steps;
    const int64_t nsub = (t1 - t0 + kSeg - 1) / kSeg;
    // states at the sub-segment starts t0, t0 + kSeg, ... (sub 0 is the checkpoint)
    const T *sub[64];
    if (nsub > 64) return GEO_ERR_ARG;
    sub[0] = (const T *)(w + Lw.off_ckpt + (size_t)seg * st);
    for (int64_t i = 1; i < nsub; ++i) {
      T *dst = (T *)(w + Lw.off_sub + (size_t)(i - 1) * st);
      const int rc = run_chain(dt, sub[i - 1], pmask, dst, H64, W64, W64, conn, op, MODE_CHAIN, kSeg, nullptr, s,
                               batch);
      if (rc != GEO_OK) return rc;
      sub[i] = dst;
    }
    for (int64_t i = nsub - 1; i >= 0; --i) {
      const int64_t a = t0 + i * kSeg;
      const int S = (int)((a + kSeg < t1) ? kSeg : t1 - a);
      T *gnext;
      int64_t gnext_pitch;
      if (a == 0) {
        gnext = grad_marker;
        gnext_pitch = pitch;
      } else {
        gnext = gbuf[gsel];
        gnext_pitch = W64;
        gsel ^= 1;
      }
      const int first = (a + S == steps);
      const int rc = launch_seg<T, TT>(op, conn, sub[i], mask, pitch, gcur, gcur_pitch, gnext, gnext_pitch, grad_mask,
                                       pitch, H, W, batch, S, first, s);
      if (rc != GEO_OK) return rc;
      gcur = gnext;
      gcur_pitch = gnext_pitch;
    }
  }
  return cudaGetLastError() == cudaSuccess ? GEO_OK : GEO_ERR_CUDA;
}

bool ok_dtype(int dt) { return dt == GEO_F32 || dt == GEO_F64; }

}  // namespace
}  // namespace geo

using namespace geo;

extern "C" {

size_t geo_chain_backward_workspace_size(geo_dtype dtype, int64_t height, int64_t width, int64_t steps,
                                         int ckpt_interval, int batch) {
  if (!ok_dtype(dtype) || height < 0 || width < 0 || steps < 0 || ckpt_interval < 1 || ckpt_interval > 512 ||
      batch < 1)
    return 0;
  return layout(dtype == GEO_F32 ? 4 : 8, height, width, steps, ckpt_interval, batch).total;
}

int geo_chain_fwd_ckpt(geo_dtype dtype, int op, const void *marker, const void *mask, void *out, int64_t height,
                       int64_t width, int64_t pitch, int conn, int64_t steps, int ckpt_interval, int batch,
                       void *workspace, size_t ws_bytes, void *stream) {
  if (!ok_dtype(dtype)) return GEO_ERR_DTYPE;
  if ((op != DILATE && op != ERODE) || (conn != 4 && conn != 8) || steps < 0 || ckpt_interval < 1 ||
      ckpt_interval > 512 || batch < 1 || height < 0 || width < 0 || pitch < width)
    return GEO_ERR_ARG;
  if (height == 0 || width == 0) return GEO_OK;
  if (!marker || !mask || !out || !workspace || marker == out) return GEO_ERR_ARG;
  const int es = dtype == GEO_F32 ? 4 : 8;
  const Layout Lw = layout(es, height, width, steps, ckpt_interval, batch);
  if (ws_bytes < Lw.total) return GEO_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  char *w = (char *)workspace;
  const size_t st = (Lw.ckpt_b + 255) & ~(size_t)255;
  // checkpoint 0 is the marker itself, packed (row stride = width)
  if (cudaMemcpy2DAsync(w + Lw.off_ckpt, width * es, marker, pitch * es, width * es, height * (int64_t)batch,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GEO_ERR_CUDA;
  // the chain kernels take one row stride for all images of a call, so the
  // segments run on packed copies: packed mask in state0, segments ping into
  // the checkpoint slots, the last segment lands in state1 and is copied out
  char *pmask = w + Lw.off_state0;
  if (cudaMemcpy2DAsync(pmask, width * es, mask, pitch * es, width * es, height * (int64_t)batch,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GEO_ERR_CUDA;
  for (int64_t seg = 0; seg < Lw.nseg; ++seg) {
    const int64_t t0 = seg * ckpt_interval;
    const int64_t len = (t0 + ckpt_interval < steps) ? ckpt_interval : steps - t0;
    const char *src = w + Lw.off_ckpt + (size_t)seg * st;
    char *dst = (seg + 1 < Lw.nseg) ? w + Lw.off_ckpt + (size_t)(seg + 1) * st : w + Lw.off_state1;
    int rc = run_chain(dtype, src, pmask, dst, height, width, width, conn, op, MODE_CHAIN, len, nullptr, stream, batch);
    if (rc != GEO_OK) return rc;
  }
  if (cudaMemcpy2DAsync(out, pitch * es, w + Lw.off_state1, width * es, width * es, height * (int64_t)batch,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GEO_ERR_CUDA;
  return GEO_OK;
}

// the per-step kernels index with 32-bit pixel coordinates on a 3-D grid
static bool grad_shape_ok(int64_t height, int64_t width, int batch) {
  return height <= (int64_t)65535 * 8 && width <= (int64_t)1 << 30 && batch <= 65535;
}

int geo_chain_backward(geo_dtype dtype, int op, const void *mask, const void *grad_out, void *grad_marker,
                       void *grad_mask, int64_t height, int64_t width, int64_t pitch, int conn, int64_t steps,
                       int ckpt_interval, int batch, void *workspace, void *stream) {
  if (!ok_dtype(dtype)) return GEO_ERR_DTYPE;
  if ((op != DILATE && op != ERODE) || (conn != 4 && conn != 8) || steps < 0 || ckpt_interval < 1 ||
      ckpt_interval > 512 || batch < 1 || height < 0 || width < 0 || pitch < width)
    return GEO_ERR_ARG;
  if (height == 0 || width == 0) return GEO_OK;
  if (!mask || !grad_out || !grad_marker || !grad_mask || !workspace || !grad_shape_ok(height, width, batch))
    return GEO_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == GEO_F32)
    return backward_impl<float>(dtype, op, conn, (const float *)mask, (const float *)grad_out, (float *)grad_marker,
                                (float *)grad_mask, height, width, pitch, steps, ckpt_interval, batch,
                                (const char *)workspace, s);
  return backward_impl<double>(dtype, op, conn, (const double *)mask, (const double *)grad_out, (double *)grad_marker,
                               (double *)grad_mask, height, width, pitch, steps, ckpt_interval, batch,
                               (const char *)workspace, s);
}

}  // extern "C"
