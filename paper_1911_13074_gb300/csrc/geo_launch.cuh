// Host-side launch of the tile kernel for one element type (included once per
// element-type translation unit so the three instantiations compile in parallel).
#pragma once

#include <mutex>
#include <set>
#include <tuple>

#include "geo_rr.cuh"
#include "geo_tile.cuh"

namespace geo {

// The kernel's dynamic shared-memory limit, set once per device, kernel and
// size (the attribute is a driver call; single-pass calls are short enough
// for it to show).
static inline cudaError_t set_smem_limit(void *k, int smem) {
  static std::mutex mu;
  static std::set<std::tuple<int, void *, int>> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> g(mu);
    if (done.count(std::make_tuple(dev, k, smem))) return cudaSuccess;
  }
  const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> g(mu);
    done.insert(std::make_tuple(dev, k, smem));
  }
  return e;
}

template <template <int> class EP>
static void *tile_kernel_ptr(int op, int conn) {
  if (op == DILATE) return conn == 8 ? (void *)tile_kernel<EP<DILATE>, 8> : (void *)tile_kernel<EP<DILATE>, 4>;
  return conn == 8 ? (void *)tile_kernel<EP<ERODE>, 8> : (void *)tile_kernel<EP<ERODE>, 4>;
}

template <template <int> class EP>
static int launch_tile_impl(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid, size_t smem) {
  void *k = tile_kernel_ptr<EP>(op, conn);
  if (set_smem_limit(k, (int)smem) != cudaSuccess)
    return GEO_ERR_CUDA;
  TileLaunch arg = L;
  void *args[] = {(void *)&arg};
  cudaError_t e = cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kThreads), args, smem, s);
  return e == cudaSuccess ? GEO_OK : GEO_ERR_CUDA;
}

template <template <int> class EP>
static int occupancy_impl(int op, int conn, size_t smem, int *bps) {
  void *k = tile_kernel_ptr<EP>(op, conn);
  if (set_smem_limit(k, (int)smem) != cudaSuccess)
    return GEO_ERR_CUDA;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, kThreads, smem) == cudaSuccess ? GEO_OK
                                                                                                : GEO_ERR_CUDA;
}

// TAGGABLE: whether the TAG instantiation exists for this shape (every
// uint8 shape; of float32, the default shape, which rank-code planes use)
template <template <int> class RP, bool TAGGABLE = RR<RP<DILATE>>::kTagged>
static void *rr_kernel_ptr(int op, int conn, bool tagged = false) {
  // RP is one of the single-image policies SU8 / SF32 / SF64; chains with
  // tagged planes take the TAG instantiation
  if constexpr (TAGGABLE) {
    if (tagged) {
      if (op == DILATE)
        return conn == 8 ? (void *)rr_kernel<RP<DILATE>, 8, true> : (void *)rr_kernel<RP<DILATE>, 4, true>;
      return conn == 8 ? (void *)rr_kernel<RP<ERODE>, 8, true> : (void *)rr_kernel<RP<ERODE>, 4, true>;
    }
  }
  if (op == DILATE) return conn == 8 ? (void *)rr_kernel<RP<DILATE>, 8> : (void *)rr_kernel<RP<DILATE>, 4>;
  return conn == 8 ? (void *)rr_kernel<RP<ERODE>, 8> : (void *)rr_kernel<RP<ERODE>, 4>;
}

template <template <int> class RP, bool TAGGABLE = RR<RP<DILATE>>::kTagged>
static int launch_rr_impl(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid) {
  if (L.tagged != nullptr && !TAGGABLE) return GEO_ERR_ARG;
  void *k = rr_kernel_ptr<RP, TAGGABLE>(op, conn, L.tagged != nullptr);
  const size_t smem = rr_smem_bytes<RP<DILATE>>();
  if (set_smem_limit(k, (int)smem) != cudaSuccess)
    return GEO_ERR_CUDA;
  TileLaunch arg = L;
  void *args[] = {(void *)&arg};
  cudaError_t e = cudaLaunchCooperativeKernel(k, dim3(grid), dim3(RP<DILATE>::NW * 32), args, smem, s);
  return e == cudaSuccess ? GEO_OK : GEO_ERR_CUDA;
}

template <template <int> class RP>
static int occupancy_rr_impl(int op, int conn, int *bps) {
  void *k = rr_kernel_ptr<RP>(op, conn);
  const size_t smem = rr_smem_bytes<RP<DILATE>>();
  if (set_smem_limit(k, (int)smem) != cudaSuccess)
    return GEO_ERR_CUDA;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, RP<DILATE>::NW * 32, smem) == cudaSuccess
             ? GEO_OK
             : GEO_ERR_CUDA;
}

}  // namespace geo
