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
// first. Per segment, in sub-segments of up to 8 steps:
//   * forward, first to last: a code kernel per 64x64 tile (32x32 for
//     float64) recomputes the sub-segment in shared memory from its start
//     state, on the tile plus an 8-pixel halo, and writes for each of the
//     tile's pixels one 32-bit word holding its routing code at every step
//     (4 bits a step: 0..8 = neighbour, 9 = mask) and its state at the end,
//     the start of the next sub-segment;
//   * reverse, last to first: a gather kernel per tile stages the gradient
//     and the code words on the tile plus the 8-pixel halo and replays the
//     steps in reverse there.
// The gradient and grad_mask touch global memory once per sub-segment
// instead of once per step, and no state is recomputed twice.
#include <cstdlib>
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
// helpers of the segment kernels
// ---------------------------------------------------------------------------

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

// ---------------------------------------------------------------------------
// split segment kernels: (A) the routing codes of each tile's own pixels for
// up to SS = 8 steps, packed into one 32-bit word per pixel (4 bits a step,
// step j in bits 4(j-1)..4j-1) in a global code plane; (B) the reverse
// replay of those steps from the staged code words. A tile's codes need the
// segment-start state only within SS of the tile (TT + 2 SS), against
// TT + 4 SS when one kernel computes the codes of the whole reverse region
// itself; the code plane (4 bytes a pixel) stays in L2 between the two.
// ---------------------------------------------------------------------------

constexpr int kSplitThreads = 512;          // two CTAs per SM
constexpr uint32_t kCodesNone = 0xffffffffu;  // outside the image: code 15 (routes nowhere) at every step

template <typename T, int TT, int SS>
struct SplitGeom {
  static_assert(SS <= 8, "8 steps of 4-bit codes in a 32-bit word");
  static constexpr int R = TT + 2 * SS;  // region side of both kernels
  static constexpr int NS = (R * R + kSplitThreads - 1) / kSplitThreads;  // staging rounds per thread
  static constexpr size_t f_bytes = sizeof(T) * R * R;
  static constexpr size_t c_bytes = sizeof(uint32_t) * R * R;
  static constexpr size_t a_smem = 3 * f_bytes;            // two states and the mask
  static constexpr size_t b_smem = 2 * f_bytes + c_bytes;  // two gradients and the code words
};

// The threads of a CTA as (column, chunk of rows) of a region of side R.
template <int R, int NT>
struct StripsN {
  static constexpr int NH = NT / R;
  static constexpr int RP = (R + NH - 1) / NH;
};

// (A) f0: the state at the sub-segment start (row stride W). Steps 1..S are
// recomputed on the cells within SS - j of the tile at step j. A thread owns
// the same cells (a column of a chunk of rows) at every step, so it keeps the
// codes of its tile cells in registers and writes each cell's code word once.
template <typename T, int OP, int CONN, int TT, int SS>
__global__ void __launch_bounds__(kSplitThreads, 2) seg_codes(const T *__restrict__ f0, const T *__restrict__ mask,
                                                              int64_t mpitch, uint32_t *__restrict__ codes,
                                                              T *__restrict__ f_next, int H, int W, int S) {
  using G = SplitGeom<T, TT, SS>;
  constexpr int R = G::R;
  using SP = StripsN<R, kSplitThreads>;
  extern __shared__ __align__(16) char smem[];
  T *fa = reinterpret_cast<T *>(smem);
  T *fb = reinterpret_cast<T *>(smem + G::f_bytes);
  T *ms = reinterpret_cast<T *>(smem + 2 * G::f_bytes);
  const int tid = threadIdx.x;
  const int b = blockIdx.z;
  const int ty0 = blockIdx.y * TT, tx0 = blockIdx.x * TT;
  const int oy = ty0 - SS, ox = tx0 - SS;  // region origin (global)
  const T ID = seg_ident<T, OP>();
  const T *fimg = f0 + (size_t)b * H * W;
  const T *mimg = mask + (size_t)b * H * mpitch;
  {
    // every load of the thread in flight before the first store
    T fv[G::NS], mv[G::NS];
#pragma unroll
    for (int it = 0; it < G::NS; ++it) {
      const int i = tid + it * kSplitThreads;
      const int r = i / R, c = i - r * R;
      const int y = oy + r, x = ox + c;
      const bool in = i < R * R && y >= 0 && y < H && x >= 0 && x < W;
      fv[it] = in ? fimg[(size_t)y * W + x] : ID;
      mv[it] = in ? mimg[(size_t)y * mpitch + x] : ID;
    }
#pragma unroll
    for (int it = 0; it < G::NS; ++it) {
      const int i = tid + it * kSplitThreads;
      if (i < R * R) {
        fa[i] = fv[it];
        ms[i] = mv[it];
      }
    }
  }
  __syncthreads();
  const int col = tid % R, chunk = tid / R;
  const int base = chunk * SP::RP;
  uint32_t cw[SP::RP];
#pragma unroll
  for (int q = 0; q < SP::RP; ++q) cw[q] = kCodesNone;
  T *cur = fa, *nxt = fb;
  for (int j = 1; j <= S; ++j) {
    const int lo = j, hi = R - j;
    const int c = col;
    const int r0 = max(lo, base), r1 = min(hi, base + SP::RP);
    const int sh = 4 * (j - 1);
    if (chunk < SP::NH && c >= lo && c < hi && r0 < r1) {
      RowExt<T, OP> up, mid, dn;
      up.load(cur + (r0 - 1) * R, c);
      mid.load(cur + r0 * R, c);
      auto cell = [&](int q) {
        const int r = base + q;
        dn.load(cur + (r + 1) * R, c);
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
        } else {
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
        const T mv = ms[r * R + c];
        const bool to_mask = beats<T, OP>(best, mv);
        nxt[r * R + c] = to_mask ? mv : best;
        const uint32_t code = to_mask ? kRouteMask : (uint32_t)k;
        cw[q] = (cw[q] & ~(15u << sh)) | (code << sh);
        up = mid;
        mid = dn;
      };
      if (r0 == base && r1 == base + SP::RP) {
        // a whole chunk: straight-line code, the window rotation is renaming
#pragma unroll
        for (int q = 0; q < SP::RP; ++q) cell(q);
      } else {
#pragma unroll
        for (int q = 0; q < SP::RP; ++q)
          if (base + q >= r0 && base + q < r1) cell(q);
      }
    }
    __syncthreads();
    T *tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  // the code words of the thread's tile cells, and (f_next) their state
  // after the S steps: the start of the next sub-segment
  const int x = ox + col;
  if (chunk < SP::NH && col >= SS && col < SS + TT && x < W) {
    uint32_t *cimg = codes + (size_t)b * H * W;
    T *nimg = f_next ? f_next + (size_t)b * H * W : nullptr;
#pragma unroll
    for (int q = 0; q < SP::RP; ++q) {
      const int r = base + q, y = oy + r;
      if (r >= SS && r < SS + TT && y < H) {
        cimg[(size_t)y * W + x] = cw[q];
        if (nimg) nimg[(size_t)y * W + x] = cur[r * R + col];
      }
    }
  }
}

// (B) g at t0 + S (g_in) carried back to t0 (g_out) with the code words of
// steps t0 + 1 .. t0 + S from (A); grad_mask gathers the mask-routed
// gradients in decreasing step order (written, not accumulated, when `first`).
template <typename T, int CONN, int TT, int SS>
__global__ void __launch_bounds__(kSplitThreads, 2) seg_gather(const uint32_t *__restrict__ codes,
                                                               const T *__restrict__ g_in, int64_t gi_pitch,
                                                               T *__restrict__ g_out, int64_t go_pitch,
                                                               T *__restrict__ gmask, int64_t gm_pitch, int H, int W,
                                                               int S, int first) {
  using G = SplitGeom<T, TT, SS>;
  constexpr int R = G::R;
  using SP = StripsN<R, kSplitThreads>;
  extern __shared__ __align__(16) char smem[];
  T *ga = reinterpret_cast<T *>(smem);
  T *gb = reinterpret_cast<T *>(smem + G::f_bytes);
  uint32_t *cs = reinterpret_cast<uint32_t *>(smem + 2 * G::f_bytes);
  const int tid = threadIdx.x;
  const int b = blockIdx.z;
  const int ty0 = blockIdx.y * TT, tx0 = blockIdx.x * TT;
  const int oy = ty0 - SS, ox = tx0 - SS;
  const T *gimg = g_in + (size_t)b * H * gi_pitch;
  const uint32_t *cimg = codes + (size_t)b * H * W;
  {
    T gv[G::NS];
    uint32_t cv[G::NS];
#pragma unroll
    for (int it = 0; it < G::NS; ++it) {
      const int i = tid + it * kSplitThreads;
      const int r = i / R, c = i - r * R;
      const int y = oy + r, x = ox + c;
      const bool in = i < R * R && y >= 0 && y < H && x >= 0 && x < W;
      gv[it] = in ? gimg[(size_t)y * gi_pitch + x] : T(0);
      cv[it] = in ? cimg[(size_t)y * W + x] : kCodesNone;
    }
#pragma unroll
    for (int it = 0; it < G::NS; ++it) {
      const int i = tid + it * kSplitThreads;
      if (i < R * R) {
        ga[i] = gv[it];
        cs[i] = cv[it];
      }
    }
  }
  // per thread: its fixed tile pixels' mask gradient
  constexpr int PT = (TT * TT + kSplitThreads - 1) / kSplitThreads;
  T gmacc[PT];
  T *gmimg = gmask + (size_t)b * H * gm_pitch;
#pragma unroll
  for (int e = 0; e < PT; ++e) {
    const int i = tid + e * kSplitThreads;
    const int r = i / TT, c = i - r * TT;
    const int y = ty0 + r, x = tx0 + c;
    gmacc[e] = (!first && i < TT * TT && y < H && x < W) ? gmimg[(size_t)y * gm_pitch + x] : T(0);
  }
  __syncthreads();
  const int col = tid % R, chunk = tid / R;
  T *gc = ga, *gn = gb;
  for (int j = S; j >= 1; --j) {
    const int sh = 4 * (j - 1);
#pragma unroll
    for (int e = 0; e < PT; ++e) {
      const int i = tid + e * kSplitThreads;
      const int r = SS + i / TT, c = SS + i % TT;
      if (i < TT * TT && ((cs[r * R + c] >> sh) & 15u) == kRouteMask) gmacc[e] += gc[r * R + c];
    }
    const int lo = SS - (j - 1), hi = R - lo;
    const int c = col;
    const int base = chunk * SP::RP;
    const int r0 = max(lo, base), r1 = min(hi, base + SP::RP);
    if (chunk < SP::NH && c >= lo && c < hi && r0 < r1) {
      // window of three rows (r - 1, r, r + 1) of codes and gradients at
      // columns c + 1, c, c - 1; the cell gathers, in increasing k, the
      // gradients of the neighbours routed to it: k = 0..2 from the row
      // below, 3..5 from its own row, 6..8 from the row above
      uint32_t kA[3], kB[3], kC[3];
      T gA[3], gB[3], gC[3];
      const uint32_t *crow = cs + (r0 - 1) * R + c - 1;
      const T *grow = gc + (r0 - 1) * R + c - 1;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        kA[i] = (crow[2 - i] >> sh) & 15u;
        gA[i] = grow[2 - i];
        kB[i] = (crow[R + 2 - i] >> sh) & 15u;
        gB[i] = grow[R + 2 - i];
      }
      auto cell = [&](int r) {
        const uint32_t *cn = cs + (r + 1) * R + c - 1;
        const T *gnr = gc + (r + 1) * R + c - 1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          kC[i] = (cn[2 - i] >> sh) & 15u;
          gC[i] = gnr[2 - i];
        }
        T acc = T(0);
#pragma unroll
        for (int i = 0; i < 3; ++i)
          if (in_shape<CONN>(i) && kC[i] == (uint32_t)i) acc += gC[i];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          if (in_shape<CONN>(3 + i) && kB[i] == (uint32_t)(3 + i)) acc += gB[i];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          if (in_shape<CONN>(6 + i) && kA[i] == (uint32_t)(6 + i)) acc += gA[i];
        gn[r * R + c] = acc;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          kA[i] = kB[i];
          gA[i] = gB[i];
          kB[i] = kC[i];
          gB[i] = gC[i];
        }
      };
      if (r0 == base && r1 == base + SP::RP) {
        // a whole chunk: straight-line code, the window rotation is renaming
#pragma unroll
        for (int q = 0; q < SP::RP; ++q) cell(base + q);
      } else {
        for (int r = r0; r < r1; ++r) cell(r);
      }
    }
    __syncthreads();
    T *tmp = gc;
    gc = gn;
    gn = tmp;
  }
  T *goimg = g_out + (size_t)b * H * go_pitch;
#pragma unroll
  for (int e = 0; e < PT; ++e) {
    const int i = tid + e * kSplitThreads;
    const int r = i / TT, c = i - r * TT;
    const int y = ty0 + r, x = tx0 + c;
    if (i < TT * TT && y < H && x < W) {
      goimg[(size_t)y * go_pitch + x] = gc[(SS + r) * R + SS + c];
      gmimg[(size_t)y * gm_pitch + x] = gmacc[e];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kBX * kBY) zero_plane(T *__restrict__ p, int64_t pitch, int H, int W) {
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  if (x >= W || y >= H) return;
  p[(size_t)blockIdx.z * H * pitch + (size_t)y * pitch + x] = T(0);
}

// Sub-segment length (8 codes of 4 bits fill a 32-bit word) and the tile
// side per element type: both kernels then hold two CTAs per SM (77 KB of
// shared memory each for float32).
constexpr int kSeg = 8;
constexpr int kTileF32 = 64, kTileF64 = 32;

struct Layout {
  int64_t npx;    // batch * H * W
  int64_t nseg;   // checkpoints (segments of C steps)
  int64_t nsub;   // sub-segment starts kept per segment (C / kSeg, rounded up)
  size_t ckpt_b;  // bytes of one packed state (all images)
  size_t off_ckpt, off_state0, off_state1, off_sub, off_g0, off_g1, off_codes, total;
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
  // routing codes of every sub-segment of a segment, a 32-bit word per pixel
  // each (split kernels)
  L.off_codes = L.off_g1 + st;
  L.total = L.off_codes + up((size_t)L.npx * sizeof(uint32_t)) * (size_t)L.nsub;
  return L;
}

template <typename T, int TT>
int launch_codes(int op, int conn, const T *f0, const T *mask, int64_t mpitch, uint32_t *codes, T *f_next, int H,
                 int W, int batch, int S, cudaStream_t s) {
  using Gm = SplitGeom<T, TT, kSeg>;
  const dim3 grid((unsigned)((W + TT - 1) / TT), (unsigned)((H + TT - 1) / TT), (unsigned)batch);
  void (*ka)(const T *, const T *, int64_t, uint32_t *, T *, int, int, int);
  if (op == DILATE) ka = conn == 8 ? seg_codes<T, DILATE, 8, TT, kSeg> : seg_codes<T, DILATE, 4, TT, kSeg>;
  else ka = conn == 8 ? seg_codes<T, ERODE, 8, TT, kSeg> : seg_codes<T, ERODE, 4, TT, kSeg>;
  if (cudaFuncSetAttribute((const void *)ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::a_smem) !=
      cudaSuccess)
    return GEO_ERR_CUDA;
  ka<<<grid, kSplitThreads, Gm::a_smem, s>>>(f0, mask, mpitch, codes, f_next, H, W, S);
  return cudaGetLastError() == cudaSuccess ? GEO_OK : GEO_ERR_CUDA;
}

template <typename T, int TT>
int launch_gather(int conn, const uint32_t *codes, const T *gin, int64_t gi_pitch, T *gout, int64_t go_pitch, T *gm,
                  int64_t gm_pitch, int H, int W, int batch, int S, int first, cudaStream_t s) {
  using Gm = SplitGeom<T, TT, kSeg>;
  const dim3 grid((unsigned)((W + TT - 1) / TT), (unsigned)((H + TT - 1) / TT), (unsigned)batch);
  void (*kb)(const uint32_t *, const T *, int64_t, T *, int64_t, T *, int64_t, int, int, int, int) =
      conn == 8 ? seg_gather<T, 8, TT, kSeg> : seg_gather<T, 4, TT, kSeg>;
  if (cudaFuncSetAttribute((const void *)kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::b_smem) !=
      cudaSuccess)
    return GEO_ERR_CUDA;
  kb<<<grid, kSplitThreads, Gm::b_smem, s>>>(codes, gin, gi_pitch, gout, go_pitch, gm, gm_pitch, H, W, S, first);
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
  T *gbuf[2] = {(T *)(w + Lw.off_g0), (T *)(w + Lw.off_g1)};
  const T *gcur = grad_out;  // the gradient being propagated and its row stride
  int64_t gcur_pitch = pitch;
  int gsel = 0;
  const size_t cst = (((size_t)Lw.npx * sizeof(uint32_t)) + 255) & ~(size_t)255;
  for (int64_t seg = Lw.nseg - 1; seg >= 0; --seg) {
    const int64_t t0 = seg * C;
    const int64_t t1 = (t0 + C < steps) ? t0 + C : steps;
    const int64_t nsub = (t1 - t0 + kSeg - 1) / kSeg;
    // states at the sub-segment starts t0, t0 + kSeg, ... (sub 0 is the checkpoint)
    const T *sub[64];
    if (nsub > 64) return GEO_ERR_ARG;
    sub[0] = (const T *)(w + Lw.off_ckpt + (size_t)seg * st);
    // forward over the segment: each code pass writes its sub-segment's
    // code words and the next sub-segment's start state
    for (int64_t i = 0; i < nsub; ++i) {
      const int64_t a = t0 + i * kSeg;
      const int S = (int)((a + kSeg < t1) ? kSeg : t1 - a);
      T *next = (i + 1 < nsub) ? (T *)(w + Lw.off_sub + (size_t)i * st) : nullptr;
      const int rc = launch_codes<T, TT>(op, conn, sub[i], mask, pitch, (uint32_t *)(w + Lw.off_codes + i * cst),
                                         next, H, W, batch, S, s);
      if (rc != GEO_OK) return rc;
      if (next) sub[i + 1] = next;
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
      const int rc = launch_gather<T, TT>(conn, (const uint32_t *)(w + Lw.off_codes + i * cst), gcur, gcur_pitch,
                                          gnext, gnext_pitch, grad_mask, pitch, H, W, batch, S, first, s);
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
