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
// first; per segment it recomputes the states forward from the checkpoint,
// keeping one routing byte per pixel and step (0..8 = neighbour, 9 = mask),
// then replays the segment's steps in reverse.
#include <cstring>

#include "geo_common.cuh"

namespace geo {
namespace {

constexpr uint8_t kRouteMask = 9;

template <int CONN>
__device__ __forceinline__ bool in_shape(int k) {
  return CONN == 8 || k == 1 || k == 3 || k == 4 || k == 5 || k == 7;
}

// Launch shape of the per-step kernels: one thread per pixel, a 32 x 8
// block of a row band, blockIdx.z = image of the batch.
constexpr int kBX = 32, kBY = 8;

// One recomputed forward step with routing codes. f, fo and code are packed
// (row stride W); the mask has the caller's row stride.
template <typename T, int OP, int CONN>
__global__ void __launch_bounds__(kBX * kBY) route_step(const T *__restrict__ f, const T *__restrict__ mask,
                                                        T *__restrict__ fo, uint8_t *__restrict__ code, int H, int W,
                                                        int64_t mpitch) {
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  if (x >= W || y >= H) return;
  const size_t img = (size_t)blockIdx.z * H * W;
  const T *fb = f + img;
  T best = T(0);
  int bk = -1;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    if (!in_shape<CONN>(k)) continue;
    const int qy = y + k / 3 - 1, qx = x + k % 3 - 1;
    if (qy < 0 || qy >= H || qx < 0 || qx >= W) continue;  // clipped neighbourhood
    const T v = fb[qy * W + qx];
    if (bk < 0 || (OP == DILATE ? (v > best) : (v < best))) {
      best = v;
      bk = k;
    }
  }
  const T mv = mask[(size_t)blockIdx.z * H * mpitch + (size_t)y * mpitch + x];
  const bool to_mask = (OP == DILATE) ? (mv < best) : (mv > best);
  const size_t i = img + (size_t)y * W + x;
  fo[i] = to_mask ? mv : best;
  code[i] = to_mask ? kRouteMask : (uint8_t)bk;
}

// One reverse step: g_out = gather of g_in along the routing codes; the mask
// gradient accumulates g_in where the code selects the mask (zero_mask: this
// is the first reverse step, so it is written instead). Row strides: g_in
// gi_pitch, g_out go_pitch, grad_mask gm_pitch (elements); codes packed.
template <typename T, int CONN>
__global__ void __launch_bounds__(kBX * kBY) gather_step(const T *__restrict__ g_in, int64_t gi_pitch,
                                                         const uint8_t *__restrict__ code, T *__restrict__ g_out,
                                                         int64_t go_pitch, T *__restrict__ gmask, int64_t gm_pitch,
                                                         int H, int W, int zero_mask) {
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  if (x >= W || y >= H) return;
  const uint8_t *cb = code + (size_t)blockIdx.z * H * W;
  const T *gb = g_in + (size_t)blockIdx.z * H * gi_pitch;
  T acc = T(0);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    if (!in_shape<CONN>(k)) continue;
    // the pixel p = q - d_k, if routed to its neighbour k, lands on q
    const int py = y - (k / 3 - 1), px = x - (k % 3 - 1);
    if (py < 0 || py >= H || px < 0 || px >= W) continue;
    if (cb[py * W + px] == k) acc += gb[(size_t)py * gi_pitch + px];
  }
  T *gm = gmask + (size_t)blockIdx.z * H * gm_pitch + (size_t)y * gm_pitch + x;
  const bool to_mask = cb[y * W + x] == kRouteMask;
  if (zero_mask) *gm = to_mask ? gb[(size_t)y * gi_pitch + x] : T(0);
  else if (to_mask) *gm += gb[(size_t)y * gi_pitch + x];
  g_out[(size_t)blockIdx.z * H * go_pitch + (size_t)y * go_pitch + x] = acc;
}

template <typename T>
__global__ void __launch_bounds__(kBX * kBY) zero_plane(T *__restrict__ p, int64_t pitch, int H, int W) {
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  if (x >= W || y >= H) return;
  p[(size_t)blockIdx.z * H * pitch + (size_t)y * pitch + x] = T(0);
}

struct Layout {
  int64_t npx;       // batch * H * W
  int64_t nseg;      // checkpoints (segments)
  size_t ckpt_b;     // bytes of one packed state (all images)
  size_t off_ckpt, off_state0, off_state1, off_code, off_g0, off_g1, total;
};

Layout layout(int es, int64_t H, int64_t W, int64_t steps, int C, int batch) {
  Layout L{};
  L.npx = (int64_t)batch * H * W;
  L.nseg = steps > 0 ? (steps + C - 1) / C : 1;
  L.ckpt_b = (size_t)L.npx * es;
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t st = up(L.ckpt_b);
  L.off_ckpt = 0;
  L.off_state0 = L.off_ckpt + st * (size_t)L.nseg;
  L.off_state1 = L.off_state0 + st;
  L.off_code = L.off_state1 + st;
  L.off_g0 = L.off_code + up((size_t)L.npx * (size_t)C);
  L.off_g1 = L.off_g0 + st;
  L.total = L.off_g1 + st;
  return L;
}

dim3 step_grid(int64_t H, int64_t W, int batch) {
  return dim3((unsigned)((W + kBX - 1) / kBX), (unsigned)((H + kBY - 1) / kBY), (unsigned)batch);
}

template <typename T>
int backward_impl(int op, int conn, const T *mask, const T *grad_out, T *grad_marker, T *grad_mask, int64_t H64,
                  int64_t W64, int64_t pitch, int64_t steps, int C, int batch, const char *ws, cudaStream_t s) {
  const Layout Lw = layout((int)sizeof(T), H64, W64, steps, C, batch);
  const int64_t n = Lw.npx;
  const int H = (int)H64, W = (int)W64;
  const dim3 grid = step_grid(H64, W64, batch), block(kBX, kBY);
  if (steps == 0) {
    zero_plane<T><<<grid, block, 0, s>>>(grad_mask, pitch, H, W);
    if (cudaMemcpy2DAsync(grad_marker, pitch * sizeof(T), grad_out, pitch * sizeof(T), W64 * sizeof(T),
                          H64 * (int64_t)batch, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return GEO_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? GEO_OK : GEO_ERR_CUDA;
  }
  char *w = const_cast<char *>(ws);
  T *st[2] = {(T *)(w + Lw.off_state0), (T *)(w + Lw.off_state1)};
  uint8_t *code = (uint8_t *)(w + Lw.off_code);
  T *gbuf[2] = {(T *)(w + Lw.off_g0), (T *)(w + Lw.off_g1)};
  // the gradient being propagated: (pointer, row stride)
  const T *gcur = grad_out;
  int64_t gcur_pitch = pitch;
  int gsel = 0;
  for (int64_t seg = Lw.nseg - 1; seg >= 0; --seg) {
    const int64_t t0 = seg * C;
    const int64_t t1 = (t0 + C < steps) ? t0 + C : steps;
    // recompute the segment's routing codes from its checkpoint
    const T *fcur = (const T *)(w + Lw.off_ckpt + (size_t)seg * ((Lw.ckpt_b + 255) & ~(size_t)255));
    for (int64_t t = t0 + 1; t <= t1; ++t) {
      T *fnext = st[(t - t0 - 1) & 1];
      uint8_t *ct = code + (size_t)(t - t0 - 1) * (size_t)n;
      if (op == DILATE) {
        if (conn == 8) route_step<T, DILATE, 8><<<grid, block, 0, s>>>(fcur, mask, fnext, ct, H, W, pitch);
        else route_step<T, DILATE, 4><<<grid, block, 0, s>>>(fcur, mask, fnext, ct, H, W, pitch);
      } else {
        if (conn == 8) route_step<T, ERODE, 8><<<grid, block, 0, s>>>(fcur, mask, fnext, ct, H, W, pitch);
        else route_step<T, ERODE, 4><<<grid, block, 0, s>>>(fcur, mask, fnext, ct, H, W, pitch);
      }
      fcur = fnext;
    }
    // replay the segment's steps in reverse
    for (int64_t t = t1; t > t0; --t) {
      const uint8_t *ct = code + (size_t)(t - t0 - 1) * (size_t)n;
      T *gnext;
      int64_t gnext_pitch;
      if (t == 1) {
        gnext = grad_marker;
        gnext_pitch = pitch;
      } else {
        gnext = gbuf[gsel];
        gnext_pitch = W;
        gsel ^= 1;
      }
      const int first = (t == steps);
      if (conn == 8)
        gather_step<T, 8><<<grid, block, 0, s>>>(gcur, gcur_pitch, ct, gnext, gnext_pitch, grad_mask, pitch, H, W,
                                                 first);
      else
        gather_step<T, 4><<<grid, block, 0, s>>>(gcur, gcur_pitch, ct, gnext, gnext_pitch, grad_mask, pitch, H, W,
                                                 first);
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
  if (!ok_dtype(dtype) || height < 0 || width < 0 || steps < 0 || ckpt_interval < 1 || batch < 1) return 0;
  return layout(dtype == GEO_F32 ? 4 : 8, height, width, steps, ckpt_interval, batch).total;
}

int geo_chain_fwd_ckpt(geo_dtype dtype, int op, const void *marker, const void *mask, void *out, int64_t height,
                       int64_t width, int64_t pitch, int conn, int64_t steps, int ckpt_interval, int batch,
                       void *workspace, size_t ws_bytes, void *stream) {
  if (!ok_dtype(dtype)) return GEO_ERR_DTYPE;
  if ((op != DILATE && op != ERODE) || (conn != 4 && conn != 8) || steps < 0 || ckpt_interval < 1 || batch < 1 ||
      height < 0 || width < 0 || pitch < width)
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
  if ((op != DILATE && op != ERODE) || (conn != 4 && conn != 8) || steps < 0 || ckpt_interval < 1 || batch < 1 ||
      height < 0 || width < 0 || pitch < width)
    return GEO_ERR_ARG;
  if (height == 0 || width == 0) return GEO_OK;
  if (!mask || !grad_out || !grad_marker || !grad_mask || !workspace || !grad_shape_ok(height, width, batch))
    return GEO_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == GEO_F32)
    return backward_impl<float>(op, conn, (const float *)mask, (const float *)grad_out, (float *)grad_marker,
                                (float *)grad_mask, height, width, pitch, steps, ckpt_interval, batch,
                                (const char *)workspace, s);
  return backward_impl<double>(op, conn, (const double *)mask, (const double *)grad_out, (double *)grad_marker,
                               (double *)grad_mask, height, width, pitch, steps, ckpt_interval, batch,
                               (const char *)workspace, s);
}

}  // extern "C"
