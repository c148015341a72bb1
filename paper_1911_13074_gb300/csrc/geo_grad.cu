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

// Identity of the neighbourhood extreme: what cells outside the image hold
// (image and mask) in the shared-memory regions, so that they never win an
// extreme, stay at the identity step after step (the mask clamp keeps them
// there) and never receive a gradient.
template <typename T, int OP>
__device__ __forceinline__ T seg_ident() {
  if (sizeof(T) == 4) return (T)(OP == DILATE ? __int_as_float(0xff800000) : __int_as_float(0x7f800000));
  return (T)(OP == DILATE ? __longlong_as_double((long long)0xfff0000000000000ULL)
                          : __longlong_as_double(0x7ff0000000000000LL));
}

template <typename T, int OP>
__device__ __forceinline__ bool beats(T v, T best) {
  return OP == DILATE ? (v > best) : (v < best);
}

// Row extreme of one row at columns c-1, c, c+1 with the lowest dx on ties
// (a = 0, 1, 2), and the centre value (the cross uses only the centre of
// the rows above and below).
template <typename T, int OP>
struct RowExt {
  T m, ctr;
  int a;
  __device__ __forceinline__ void load(const T *row, int c) {
    const T v0 = row[c - 1], v1 = row[c], v2 = row[c + 1];
    m = v0;
    a = 0;
    if (beats<T, OP>(v1, m)) {
      m = v1;
      a = 1;
    }
    if (beats<T, OP>(v2, m)) {
      m = v2;
      a = 2;
    }
    ctr = v1;
  }
};

// The threads of a CTA as (column, chunk of rows) of a region of side R:
// thread t takes column t % R and rows [chunk * RP, chunk * RP + RP).
template <int R>
struct Strips {
  static constexpr int NH = kSegThreads / R;        // chunks
  static constexpr int RP = (R + NH - 1) / NH;      // rows per chunk
};

// f0: the state at the segment start, packed (row stride W). S <= SS steps
// t0+1 .. t0+S are recomputed; then g at t0+S (g_in) is carried back to t0
// (g_out) and grad_mask gathers the mask-routed gradients of those steps in
// decreasing step order (written, not accumulated, when `first`).
//
// Forward: every thread walks one column over its chunk of rows with a
// sliding window of three row extremes, so each row extreme (and its lowest
// dx) is computed once and used by three cells; the cell's neighbourhood
// extreme is the first of the rows above / at / below that attains the
// largest row extreme, which is the lowest index k = (dy+1)*3 + (dx+1) in
// row-major order. Reverse: the same walk with a window of three rows of
// routing codes and gradients; each cell adds the gradients routed to it in
// increasing k.
template <typename T, int OP, int CONN, int TT, int SS>
__global__ void __launch_bounds__(kSegThreads) seg_backward(const T *__restrict__ f0, const T *__restrict__ mask,
                                                            int64_t mpitch, const T *__restrict__ g_in,
                                                            int64_t gi_pitch, T *__restrict__ g_out, int64_t go_pitch,
                                                            T *__restrict__ gmask, int64_t gm_pitch, int H, int W,
                                                            int S, int first) {
  using G = SegGeom<T, TT, SS>;
  constexpr int RF = G::RF, RB = G::RB;
  using SF = Strips<RF>;
  using SB = Strips<RB>;
  extern __shared__ __align__(16) char smem[];
  T *fa = reinterpret_cast<T *>(smem);
  T *fb = reinterpret_cast<T *>(smem + G::f_bytes);
  T *ms = reinterpret_cast<T *>(smem + 2 * G::f_bytes);
  uint8_t *codes = reinterpret_cast<uint8_t *>(smem + 3 * G::f_bytes);
  T *ga = reinterpret_cast<T *>(smem + 3 * G::f_bytes + G::code_bytes);
  T *gb = reinterpret_cast<T *>(smem + 3 * G::f_bytes + G::code_bytes + G::g_bytes);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kSegT + tx;
  const int b = blockIdx.z;
  const int ty0 = blockIdx.y * TT, tx0 = blockIdx.x * TT;
  const int fy0 = ty0 - 2 * SS, fx0 = tx0 - 2 * SS;  // forward region origin (global)
  const int by0 = ty0 - SS, bx0 = tx0 - SS;          // reverse region origin (global)
  const T ID = seg_ident<T, OP>();
  const T *fimg = f0 + (size_t)b * H * W;
  const T *mimg = mask + (size_t)b * H * mpitch;
  // stage f0 and the mask on the forward region (the identity outside the image)
  for (int r = ty; r < RF; r += kSegT) {
    const int y = fy0 + r;
    for (int c = tx; c < RF; c += kSegT) {
      const int x = fx0 + c;
      const bool in = y >= 0 && y < H && x >= 0 && x < W;
      fa[r * RF + c] = in ? fimg[(size_t)y * W + x] : ID;
      ms[r * RF + c] = in ? mimg[(size_t)y * mpitch + x] : ID;
    }
  }
  __syncthreads();
  // forward: step j computes the cells within 2SS - j of the tile and keeps
  // the routing codes of the cells within SS of it
  const int fcol = tid % RF, fchunk = tid / RF;
  T *cur = fa, *nxt = fb;
  for (int j = 1; j <= S; ++j) {
    const int lo = j, hi = RF - j;  // rows / cols [lo, hi) of the forward region
    uint8_t *ct = codes + (size_t)(j - 1) * RB * RB;
    const int c = fcol;
    const int r0 = max(lo, fchunk * SF::RP), r1 = min(hi, fchunk * SF::RP + SF::RP);
    if (fchunk < SF::NH && c >= lo && c < hi && r0 < r1) {
      RowExt<T, OP> up, mid, dn;
      up.load(cur + (r0 - 1) * RF, c);
      mid.load(cur + r0 * RF, c);
      for (int r = r0; r < r1; ++r) {
        dn.load(cur + (r + 1) * RF, c);
        T best;
        int k;
        if (CONN == 8) {
          best = up.m;
          k = up.a;
          if (beats<T, OP>(mid.m, best)) {
            best = mid.m;
            k = 3 + mid.a;
          }
          if (beats<T, OP>(dn.m, best)) {
            best = dn.m;
            k = 6 + dn.a;
          }
        } else {  // the cross: k = 1, 3, 4, 5, 7
          best = up.ctr;
          k = 1;
          if (beats<T, OP>(mid.m, best)) {
            best = mid.m;
            k = 3 + mid.a;
          }
          if (beats<T, OP>(dn.ctr, best)) {
            best = dn.ctr;
            k = 7;
          }
        }
        const T mv = ms[r * RF + c];
        const bool to_mask = beats<T, OP>(best, mv);  // mask strictly beyond the extreme
        nxt[r * RF + c] = to_mask ? mv : best;
        const int rb = r - SS, cb = c - SS;
        if (rb >= 0 && rb < RB && cb >= 0 && cb < RB) ct[rb * RB + cb] = to_mask ? kRouteMask : (uint8_t)k;
        up = mid;
        mid = dn;
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
  const int bcol = tid % RB, bchunk = tid / RB;
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
    // g at t0 + j - 1 on the cells within j - 1 of the tile: cell q gathers
    // g(p) from p = q - d_k for k = 0..8 where p routed to k; in row terms
    // k = 0..2 read the row below (columns c+1, c, c-1), k = 3..5 the own
    // row, k = 6..8 the row above
    const int lo = SS - (j - 1), hi = RB - lo;
    const int c = bcol;
    const int r0 = max(lo, bchunk * SB::RP), r1 = min(hi, bchunk * SB::RP + SB::RP);
    if (bchunk < SB::NH && c >= lo && c < hi && r0 < r1) {
      // window: codes and gradients of rows r-1 (A), r (B), r+1 (C) at columns c+1, c, c-1
      uint8_t kA[3], kB[3], kC[3];
      T gA[3], gB[3], gC[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        kA[i] = ct[(r0 - 1) * RB + c + 1 - i];
        gA[i] = gc[(r0 - 1) * RB + c + 1 - i];
        kB[i] = ct[r0 * RB + c + 1 - i];
        gB[i] = gc[r0 * RB + c + 1 - i];
      }
      for (int r = r0; r < r1; ++r) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          kC[i] = ct[(r + 1) * RB + c + 1 - i];
          gC[i] = gc[(r + 1) * RB + c + 1 - i];
        }
        T acc = T(0);
#pragma unroll
        for (int i = 0; i < 3; ++i)  // k = i: p in the row below
          if (in_shape<CONN>(i)) acc = kC[i] == i ? acc + gC[i] : acc;
#pragma unroll
        for (int i = 0; i < 3; ++i)  // k = 3 + i: the own row
          if (in_shape<CONN>(3 + i)) acc = kB[i] == 3 + i ? acc + gB[i] : acc;
#pragma unroll
        for (int i = 0; i < 3; ++i)  // k = 6 + i: the row above
          if (in_shape<CONN>(6 + i)) acc = kA[i] == 6 + i ? acc + gA[i] : acc;
        gn[r * RB + c] = acc;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          kA[i] = kB[i];
          gA[i] = gB[i];
          kB[i] = kC[i];
          gB[i] = gC[i];
        }
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
// 8 steps measured best on workload 4 (17.2 ms forward + backward; 6 steps
// 19.3 ms, 4 steps 20.6 ms: the halos shrink but launches and staging
// double); longer sub-segments do not fit 227 KB of shared memory at a
// 64-pixel tile.
#ifndef GEO_SEG_STEPS
#define GEO_SEG_STEPS 8
#endif
constexpr int kSeg = GEO_SEG_STEPS;
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
