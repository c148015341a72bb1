// Openings, closings, granulometry with its pattern spectrum, and alternating
// sequential filters (Section 2, Eq. 16-20), composed from the unmasked 3x3
// chains of the register-resident kernel (morph_window_erode / _dilate, s
// elementary steps for a (2s+1)^2 square).
//
// * gamma_s(f) = delta_s(eps_s(f)) and phi_s(f) = eps_s(delta_s(f)): two window
//   calls, the second in place on the output.
// * ASF_s = phi_s gamma_s ... phi_1 gamma_1 is the sequence of elementary
//   steps E1 D1 D1 E1 E2 D2 D2 E2 ... Es Ds Ds Es (E = eps_1, D = delta_1,
//   counts as written). Runs of the same operation are merged into one window
//   call (E1, D2, E3, D4, ..., D2s, Es): the same steps in the same order,
//   2s + 1 launches instead of 4s.
// * G_s = sum of gamma_s(f) for s = 0..smax: eps_s(f) is kept and eroded one
//   more step for each s (eps_s = eps_1 eps_{s-1} by Eq. 4's nesting), the
//   dilation of s steps goes to a second buffer, and a two-stage reduction
//   sums it in double (fixed partition and order: deterministic; exact for
//   uint8 images). PS_s = G_s - G_{s+1}.
#include <cstring>

#include "geo_common.cuh"

namespace geo {
namespace {

constexpr int kSumBlocks = 1024, kSumThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kSumThreads) sum_partial(const T *__restrict__ f, int64_t H, int64_t W,
                                                           int64_t pitch, double *__restrict__ partial) {
  // block b sums rows b, b + gridDim.x, ...; thread t columns t, t + 256, ...
  double acc = 0.0;
  for (int64_t y = blockIdx.x; y < H; y += gridDim.x) {
    const T *row = f + y * pitch;
    for (int64_t x = threadIdx.x; x < W; x += kSumThreads) acc += (double)row[x];
  }
  __shared__ double red[kSumThreads];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kSumThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// out[0] = sum of partial[0..n) in a fixed tree order (one block)
__global__ void __launch_bounds__(kSumBlocks) sum_final(const double *__restrict__ partial, int n, double *out) {
  __shared__ double red[kSumBlocks];
  red[threadIdx.x] = (int)threadIdx.x < n ? partial[threadIdx.x] : 0.0;
  __syncthreads();
  for (int o = kSumBlocks / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void spectrum(const double *__restrict__ G, double *__restrict__ PS, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) PS[i] = G[i] - G[i + 1];
}

int elem_bytes(int dt) { return dt == GEO_U8 ? 1 : dt == GEO_F32 ? 4 : 8; }

int image_sum(int dt, const void *f, int64_t H, int64_t W, int64_t pitch, double *partial, double *out,
              cudaStream_t s) {
  const int nb = (int)(H < kSumBlocks ? H : kSumBlocks);
  if (dt == GEO_U8) sum_partial<uint8_t><<<nb, kSumThreads, 0, s>>>((const uint8_t *)f, H, W, pitch, partial);
  else if (dt == GEO_F32) sum_partial<float><<<nb, kSumThreads, 0, s>>>((const float *)f, H, W, pitch, partial);
  else sum_partial<double><<<nb, kSumThreads, 0, s>>>((const double *)f, H, W, pitch, partial);
  sum_final<<<1, kSumBlocks, 0, s>>>(partial, nb, out);
  return cudaGetLastError() == cudaSuccess ? GEO_OK : GEO_ERR_CUDA;
}

int window(int op, int dt, const void *in, void *out, int64_t H, int64_t W, int64_t pitch, int64_t s, void *stream) {
  return op == ERODE ? morph_window_erode((geo_dtype)dt, in, out, H, W, pitch, s, stream)
                     : morph_window_dilate((geo_dtype)dt, in, out, H, W, pitch, s, stream);
}

bool valid_dtype(int dt) { return dt == GEO_U8 || dt == GEO_F32 || dt == GEO_F64; }

bool overlap(const void *a, const void *b, size_t n) {
  const char *x = (const char *)a, *y = (const char *)b;
  return x < y + n && y < x + n;
}

// opening (first = ERODE) or closing (first = DILATE) of half size s
int open_close(int first, geo_dtype dt, const void *f, void *out, int64_t H, int64_t W, int64_t pitch, int64_t s,
               void *stream) {
  if (!valid_dtype(dt)) return GEO_ERR_DTYPE;
  if (H < 0 || W < 0 || pitch < W || s < 0) return GEO_ERR_ARG;
  if (H == 0 || W == 0) return GEO_OK;
  if (!f || !out) return GEO_ERR_ARG;
  const size_t span = (size_t)((H - 1) * pitch + W) * elem_bytes(dt);
  if (f != out && overlap(f, out, span)) return GEO_ERR_ARG;
  int rc = window(first, dt, f, out, H, W, pitch, s, stream);
  if (rc == GEO_OK) rc = window(first == ERODE ? DILATE : ERODE, dt, out, out, H, W, pitch, s, stream);
  return rc;
}

}  // namespace
}  // namespace geo

using namespace geo;

extern "C" {

int geo_opening(geo_dtype dtype, const void *f, void *out, int64_t height, int64_t width, int64_t pitch,
                int64_t half_size, void *stream) {
  return open_close(ERODE, dtype, f, out, height, width, pitch, half_size, stream);
}

int geo_closing(geo_dtype dtype, const void *f, void *out, int64_t height, int64_t width, int64_t pitch,
                int64_t half_size, void *stream) {
  return open_close(DILATE, dtype, f, out, height, width, pitch, half_size, stream);
}

int geo_asf(geo_dtype dtype, const void *f, void *out, int64_t height, int64_t width, int64_t pitch, int64_t s,
            void *stream) {
  if (!valid_dtype(dtype)) return GEO_ERR_DTYPE;
  const int64_t H = height, W = width;
  if (H < 0 || W < 0 || pitch < W || s < 0) return GEO_ERR_ARG;
  if (H == 0 || W == 0) return GEO_OK;
  if (!f || !out) return GEO_ERR_ARG;
  const int es = elem_bytes(dtype);
  const size_t span = (size_t)((H - 1) * pitch + W) * es;
  if (f != out && overlap(f, out, span)) return GEO_ERR_ARG;
  if (s == 0) {
    if (f == out) return GEO_OK;
    return cudaMemcpy2DAsync(out, pitch * es, f, pitch * es, W * es, H, cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream) == cudaSuccess
               ? GEO_OK
               : GEO_ERR_CUDA;
  }
  // level k contributes the runs E k, D k, D k, E k; equal neighbours merge,
  // which leaves E 1, D 2, E 3, D 4, ..., D 2s, E s
  int rc = GEO_OK;
  const void *src = f;
  int cur_op = ERODE;
  int64_t run = 0;
  auto flush = [&](int op, int64_t n) {
    if (rc != GEO_OK || n == 0) return;
    rc = window(op, dtype, src, out, H, W, pitch, n, stream);
    src = out;
  };
  for (int64_t k = 1; k <= s; ++k) {
    const int seq[4] = {ERODE, DILATE, DILATE, ERODE};
    for (int i = 0; i < 4; ++i) {
      if (seq[i] == cur_op) {
        run += k;
      } else {
        flush(cur_op, run);
        cur_op = seq[i];
        run = k;
      }
    }
  }
  flush(cur_op, run);
  return rc;
}

int geo_granulometry(geo_dtype dtype, const void *f, int64_t height, int64_t width, int64_t pitch, int64_t smax,
                     double *G, double *PS, void *stream) {
  if (!valid_dtype(dtype)) return GEO_ERR_DTYPE;
  const int64_t H = height, W = width;
  if (H < 0 || W < 0 || pitch < W || smax < 0) return GEO_ERR_ARG;
  if (!G) return GEO_ERR_ARG;
  if (((uintptr_t)G % 8) || (PS && ((uintptr_t)PS % 8))) return GEO_ERR_ALIGN;
  cudaStream_t s = (cudaStream_t)stream;
  if (H == 0 || W == 0) {
    if (cudaMemsetAsync(G, 0, (size_t)(smax + 1) * sizeof(double), s) != cudaSuccess) return GEO_ERR_CUDA;
    if (PS && smax > 0 && cudaMemsetAsync(PS, 0, (size_t)smax * sizeof(double), s) != cudaSuccess)
      return GEO_ERR_CUDA;
    return GEO_OK;
  }
  if (!f) return GEO_ERR_ARG;
  const int es = elem_bytes(dtype);
  // scratch: [partial sums][eps_s(f)][gamma_s(f)], images with f's pitch
  const size_t part_b = kSumBlocks * sizeof(double);
  const size_t img_b = (((size_t)((H - 1) * pitch + W) * es) + 255) / 256 * 256;
  void *scratch = nullptr;
  int rc = pool_alloc(&scratch, part_b + 2 * img_b, s);
  if (rc != GEO_OK) return rc;
  double *partial = (double *)scratch;
  char *ero = (char *)scratch + part_b, *gam = ero + img_b;
  rc = image_sum(dtype, f, H, W, pitch, partial, G, s);
  for (int64_t k = 1; k <= smax && rc == GEO_OK; ++k) {
    rc = window(ERODE, dtype, k == 1 ? f : ero, ero, H, W, pitch, 1, stream);
    if (rc == GEO_OK) rc = window(DILATE, dtype, ero, gam, H, W, pitch, k, stream);
    if (rc == GEO_OK) rc = image_sum(dtype, gam, H, W, pitch, partial, G + k, s);
  }
  if (rc == GEO_OK && PS && smax > 0) {
    spectrum<<<(unsigned)((smax + 255) / 256), 256, 0, s>>>(G, PS, smax);
    if (cudaGetLastError() != cudaSuccess) rc = GEO_ERR_CUDA;
  }
  if (pool_free(scratch, s) != GEO_OK && rc == GEO_OK) rc = GEO_ERR_CUDA;
  return rc;
}

}  // extern "C"
