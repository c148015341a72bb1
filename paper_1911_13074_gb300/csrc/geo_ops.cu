// Geodesic operators of Section 2 built on reconstruction (Eq. 6-12):
// h-maxima, dome extraction, hole filling, removal of border objects, and
// opening by reconstruction. Each is a few elementwise kernels around the
// reconstruction driver (run_chain, MODE_REC) or the window chain.
//
// Arithmetic that produces pixel values (the h-maxima marker f - h, and the
// differences of DOME and RAOBJ) is done in the image's element type: uint8
// saturates at 0, float32 rounds to float32, float64 to float64.
#include <cmath>

#include "geo_common.cuh"

namespace geo {
namespace {

constexpr int kEX = 32, kEY = 8;  // elementwise kernels: 32 x 8 blocks

dim3 egrid(int64_t H, int64_t W) { return dim3((unsigned)((W + kEX - 1) / kEX), (unsigned)((H + kEY - 1) / kEY)); }

template <typename T>
__device__ __forceinline__ T sub_elem(T a, T b) {
  return a - b;
}
template <>
__device__ __forceinline__ uint8_t sub_elem<uint8_t>(uint8_t a, uint8_t b) {
  return a > b ? (uint8_t)(a - b) : (uint8_t)0;  // saturating
}

// out = f - h (element type; uint8 saturates at 0)
template <typename T>
__global__ void marker_sub(const T *__restrict__ f, T *__restrict__ out, int64_t H, int64_t W, int64_t pitch, T h) {
  const int64_t x = blockIdx.x * (int64_t)kEX + threadIdx.x, y = blockIdx.y * (int64_t)kEY + threadIdx.y;
  if (x >= W || y >= H) return;
  out[y * pitch + x] = sub_elem<T>(f[y * pitch + x], h);
}

// out = a - b (element type); b may alias out
template <typename T>
__global__ void image_sub(const T *__restrict__ a, const T *b, T *out, int64_t H, int64_t W, int64_t pitch) {
  const int64_t x = blockIdx.x * (int64_t)kEX + threadIdx.x, y = blockIdx.y * (int64_t)kEY + threadIdx.y;
  if (x >= W || y >= H) return;
  out[y * pitch + x] = sub_elem<T>(a[y * pitch + x], b[y * pitch + x]);
}

// order-preserving integer keys of the element types, for atomic extremes
__device__ __forceinline__ long long key_of(uint8_t v) { return v; }
__device__ __forceinline__ long long key_of(float v) {
  const int b = __float_as_int(v);
  return b >= 0 ? b : (b ^ 0x7fffffff);
}
__device__ __forceinline__ long long key_of(double v) {
  const long long b = __double_as_longlong(v);
  return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ void from_key(long long k, uint8_t &v) { v = (uint8_t)k; }
__device__ __forceinline__ void from_key(long long k, float &v) {
  const int b = (int)k;
  v = __int_as_float(b >= 0 ? b : (b ^ 0x7fffffff));
}
__device__ __forceinline__ void from_key(long long k, double &v) {
  v = __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffLL));
}

__global__ void key_init(long long *key, long long v) { *key = v; }

// global maximum (MAX) or minimum of the image's keys into *key
template <typename T, bool MAX>
__global__ void reduce_key(const T *__restrict__ f, int64_t H, int64_t W, int64_t pitch, long long *key) {
  const int64_t x = blockIdx.x * (int64_t)kEX + threadIdx.x, y = blockIdx.y * (int64_t)kEY + threadIdx.y;
  long long k = MAX ? (long long)0x8000000000000000ULL : 0x7fffffffffffffffLL;
  if (x < W && y < H) k = key_of(f[y * pitch + x]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long q = __shfl_xor_sync(0xffffffffu, k, o);
    k = MAX ? (q > k ? q : k) : (q < k ? q : k);
  }
  if ((threadIdx.x & 31) == 0) {
    if (MAX) atomicMax(key, k);
    else atomicMin(key, k);
  }
}

// out = f on the border pixels, the value of *key elsewhere
template <typename T>
__global__ void border_marker(const T *__restrict__ f, T *__restrict__ out, int64_t H, int64_t W, int64_t pitch,
                              const long long *key) {
  const int64_t x = blockIdx.x * (int64_t)kEX + threadIdx.x, y = blockIdx.y * (int64_t)kEY + threadIdx.y;
  if (x >= W || y >= H) return;
  T fill;
  from_key(*key, fill);
  const bool border = (y == 0 || x == 0 || y == H - 1 || x == W - 1);
  out[y * pitch + x] = border ? f[y * pitch + x] : fill;
}

int check(int dt, const void *f, const void *out, int64_t H, int64_t W, int64_t pitch, int conn) {
  if (dt != GEO_U8 && dt != GEO_F32 && dt != GEO_F64) return GEO_ERR_DTYPE;
  if (H < 0 || W < 0 || pitch < W || (conn != 4 && conn != 8)) return GEO_ERR_ARG;
  if (H == 0 || W == 0) return GEO_OK;
  if (!f || !out) return GEO_ERR_ARG;
  const int es = dt == GEO_U8 ? 1 : dt == GEO_F32 ? 4 : 8;
  const size_t span = (size_t)((H - 1) * pitch * es + W * es);
  const char *a = (const char *)f, *b = (const char *)out;
  if (a < b + span && b < a + span) return GEO_ERR_ARG;  // out is written while f is the mask
  return GEO_OK;
}

template <typename T>
int hmax_impl(int dt, const T *f, T *out, int64_t H, int64_t W, int64_t pitch, int conn, double h, bool dome,
              cudaStream_t s) {
  T hv;
  if (dt == GEO_U8) {
    const double hf = std::floor(h);
    hv = (T)(hf > 255.0 ? 255.0 : hf);
  } else {
    hv = (T)h;
  }
  marker_sub<T><<<egrid(H, W), dim3(kEX, kEY), 0, s>>>(f, out, H, W, pitch, hv);
  if (cudaGetLastError() != cudaSuccess) return GEO_ERR_CUDA;
  // reconstruction in place: the marker is `out`, the mask f
  int rc = run_chain(dt, out, f, out, H, W, pitch, conn, DILATE, MODE_REC, H * W + 1 + 1024, nullptr, s, 1);
  if (rc != GEO_OK || !dome) return rc;
  image_sub<T><<<egrid(H, W), dim3(kEX, kEY), 0, s>>>(f, out, out, H, W, pitch);
  return cudaGetLastError() == cudaSuccess ? GEO_OK : GEO_ERR_CUDA;
}

template <typename T>
int border_impl(int dt, const T *f, T *out, int64_t H, int64_t W, int64_t pitch, int conn, bool fill,
                cudaStream_t s) {
  long long *key = nullptr;
  if (pool_alloc((void **)&key, sizeof(long long), s) != GEO_OK) return GEO_ERR_CUDA;
  // HFILL: the interior starts at max f (erosion by reconstruction); RAOBJ:
  // at min f (dilation by reconstruction)
  key_init<<<1, 1, 0, s>>>(key, fill ? (long long)0x8000000000000000ULL : 0x7fffffffffffffffLL);
  if (fill) reduce_key<T, true><<<egrid(H, W), dim3(kEX, kEY), 0, s>>>(f, H, W, pitch, key);
  else reduce_key<T, false><<<egrid(H, W), dim3(kEX, kEY), 0, s>>>(f, H, W, pitch, key);
  border_marker<T><<<egrid(H, W), dim3(kEX, kEY), 0, s>>>(f, out, H, W, pitch, key);
  int rc = cudaGetLastError() == cudaSuccess ? GEO_OK : GEO_ERR_CUDA;
  if (rc == GEO_OK)
    rc = run_chain(dt, out, f, out, H, W, pitch, conn, fill ? ERODE : DILATE, MODE_REC, H * W + 1 + 1024, nullptr, s,
                   1);
  if (rc == GEO_OK && !fill) {
    image_sub<T><<<egrid(H, W), dim3(kEX, kEY), 0, s>>>(f, out, out, H, W, pitch);
    if (cudaGetLastError() != cudaSuccess) rc = GEO_ERR_CUDA;
  }
  if (pool_free(key, s) != GEO_OK && rc == GEO_OK) rc = GEO_ERR_CUDA;
  return rc;
}

}  // namespace
}  // namespace geo

using namespace geo;

extern "C" {

int geo_hmax(geo_dtype dtype, const void *f, void *out, int64_t height, int64_t width, int64_t pitch, int conn,
             double h, void *stream) {
  int rc = check(dtype, f, out, height, width, pitch, conn);
  if (rc != GEO_OK || height == 0 || width == 0) return rc;
  if (!(h >= 0.0)) return GEO_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == GEO_U8) return hmax_impl<uint8_t>(dtype, (const uint8_t *)f, (uint8_t *)out, height, width, pitch, conn, h, false, s);
  if (dtype == GEO_F32) return hmax_impl<float>(dtype, (const float *)f, (float *)out, height, width, pitch, conn, h, false, s);
  return hmax_impl<double>(dtype, (const double *)f, (double *)out, height, width, pitch, conn, h, false, s);
}

int geo_dome(geo_dtype dtype, const void *f, void *out, int64_t height, int64_t width, int64_t pitch, int conn,
             double h, void *stream) {
  int rc = check(dtype, f, out, height, width, pitch, conn);
  if (rc != GEO_OK || height == 0 || width == 0) return rc;
  if (!(h >= 0.0)) return GEO_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == GEO_U8) return hmax_impl<uint8_t>(dtype, (const uint8_t *)f, (uint8_t *)out, height, width, pitch, conn, h, true, s);
  if (dtype == GEO_F32) return hmax_impl<float>(dtype, (const float *)f, (float *)out, height, width, pitch, conn, h, true, s);
  return hmax_impl<double>(dtype, (const double *)f, (double *)out, height, width, pitch, conn, h, true, s);
}

int geo_hfill(geo_dtype dtype, const void *f, void *out, int64_t height, int64_t width, int64_t pitch, int conn,
              void *stream) {
  int rc = check(dtype, f, out, height, width, pitch, conn);
  if (rc != GEO_OK || height == 0 || width == 0) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == GEO_U8) return border_impl<uint8_t>(dtype, (const uint8_t *)f, (uint8_t *)out, height, width, pitch, conn, true, s);
  if (dtype == GEO_F32) return border_impl<float>(dtype, (const float *)f, (float *)out, height, width, pitch, conn, true, s);
  return border_impl<double>(dtype, (const double *)f, (double *)out, height, width, pitch, conn, true, s);
}

int geo_raobj(geo_dtype dtype, const void *f, void *out, int64_t height, int64_t width, int64_t pitch, int conn,
              void *stream) {
  int rc = check(dtype, f, out, height, width, pitch, conn);
  if (rc != GEO_OK || height == 0 || width == 0) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == GEO_U8) return border_impl<uint8_t>(dtype, (const uint8_t *)f, (uint8_t *)out, height, width, pitch, conn, false, s);
  if (dtype == GEO_F32) return border_impl<float>(dtype, (const float *)f, (float *)out, height, width, pitch, conn, false, s);
  return border_impl<double>(dtype, (const double *)f, (double *)out, height, width, pitch, conn, false, s);
}

int geo_open_rec(geo_dtype dtype, const void *f, void *out, int64_t height, int64_t width, int64_t pitch, int conn,
                 int64_t half_size, void *stream) {
  int rc = check(dtype, f, out, height, width, pitch, conn);
  if (rc != GEO_OK || height == 0 || width == 0) return rc;
  if (half_size < 0) return GEO_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // marker: erosion by the (2s+1)^2 square (s unmasked 3x3 steps), then
  // dilation by reconstruction under f, in place
  rc = run_chain(dtype, f, nullptr, out, height, width, pitch, 8, ERODE, MODE_CHAIN, half_size, nullptr, s, 1);
  if (rc != GEO_OK) return rc;
  return run_chain(dtype, out, f, out, height, width, pitch, conn, DILATE, MODE_REC, height * width + 1 + 1024,
                   nullptr, s, 1);
}

}  // extern "C"
