// Throughput probe of the min/max forms the chains are built from, for the
// rooflines of bench.py (a path bound by plain ALU arithmetic reports against
// a peak derived from the unit rate and the clock). A mixed form counts each
// maximum once, whether it took one instruction or two.
//
// One 1024-thread block per SM (the dynamic shared memory request keeps a
// second block off), each thread running NACC independent chains of the
// packed max. The block's own clock64 span gives the lane-ops per SM clock;
// clock64 against globaltimer over the same span gives the clock.
#include <cuda_runtime.h>

#include <cstdint>

#include "geo_tile.cuh"

namespace geo {
namespace {

constexpr int kProbeAcc = 16;
constexpr int kProbeIters = 2048;
constexpr int kProbeThreads = 1024;
constexpr int kProbeSmem = 150 * 1024;

// Form 0: max.u16x2; 1: max.f16x2; 2: three-input max.f32 (the float32
// step's row and column 3-extremes); 3: a 2:1 mix of max.u16x2 and an exact
// max of u16 lanes done by f16 arithmetic on the FMA pipe (fma.relu then
// fma, two instructions), the fastest mix of two pipes measured. Chain i of
// a thread uses the second form of the mix when i % 3 == 2.
template <int FORM>
__device__ __forceinline__ void probe_op(uint32_t &a, uint32_t b, int i) {
  if constexpr (FORM == 0) {
    asm volatile("max.u16x2 %0, %0, %1;" : "+r"(a) : "r"(b));
  } else if constexpr (FORM == 1) {
    asm volatile("max.f16x2 %0, %0, %1;" : "+r"(a) : "r"(b));
  } else if constexpr (FORM == 2) {
    asm volatile("max.f32 %0, %0, %1, %0;" : "+r"(a) : "r"(b));
  } else {
    if (i % 3 != 2) {
      asm volatile("max.u16x2 %0, %0, %1;" : "+r"(a) : "r"(b));
    } else {
      uint32_t r;
      asm volatile("fma.rn.relu.f16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(b), "r"(0xBC00BC00u), "r"(a));
      asm volatile("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(a) : "r"(r), "r"(0x3C003C00u), "r"(b));
    }
  }
}

template <int FORM>
__global__ void __launch_bounds__(kProbeThreads, 1) probe_kernel(unsigned long long *rec, uint32_t *sink) {
  uint32_t a[kProbeAcc];
#pragma unroll
  for (int i = 0; i < kProbeAcc; ++i) a[i] = (threadIdx.x * 7u + (uint32_t)i) & 0x00ff00ffu;
  const uint32_t b = (threadIdx.x * 13u) & 0x00ff00ffu;
  __syncthreads();
  const unsigned long long c0 = clock64(), g0 = globaltimer_ns();
#pragma unroll 1
  for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
    for (int i = 0; i < kProbeAcc; ++i) probe_op<FORM>(a[i], b, i);
  }
  __syncthreads();
  const unsigned long long c1 = clock64(), g1 = globaltimer_ns();
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kProbeAcc; ++i) s ^= a[i];
  if (s == 0x12345678u) sink[blockIdx.x] = s;  // keeps the chains live
  if (threadIdx.x == 0) {
    rec[2 * blockIdx.x] = c1 - c0;
    rec[2 * blockIdx.x + 1] = g1 - g0;
  }
}

template <int FORM>
int run_probe(int nsm, cudaStream_t st, double *rate, double *mhz) {
  unsigned long long *rec = nullptr;
  uint32_t *sink = nullptr;
  // stream-ordered: no device-wide synchronisation around the probe
  if (cudaMallocAsync(&rec, sizeof(unsigned long long) * 2 * nsm, st) != cudaSuccess) return GEO_ERR_CUDA;
  if (cudaMallocAsync(&sink, sizeof(uint32_t) * nsm, st) != cudaSuccess) {
    cudaFreeAsync(rec, st);
    return GEO_ERR_CUDA;
  }
  int rc = GEO_OK;
  unsigned long long *h = new unsigned long long[2 * (size_t)nsm];
  if (cudaFuncSetAttribute(probe_kernel<FORM>, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem) !=
      cudaSuccess)
    rc = GEO_ERR_CUDA;
  for (int rep = 0; rc == GEO_OK && rep < 3; ++rep) {  // the last of three launches is kept
    probe_kernel<FORM><<<nsm, kProbeThreads, kProbeSmem, st>>>(rec, sink);
    if (cudaGetLastError() != cudaSuccess) rc = GEO_ERR_CUDA;
  }
  if (rc == GEO_OK &&
      (cudaMemcpyAsync(h, rec, sizeof(unsigned long long) * 2 * nsm, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    rc = GEO_ERR_CUDA;
  if (rc == GEO_OK) {
    double cyc = 0, ns = 0;
    for (int i = 0; i < nsm; ++i) {
      cyc += (double)h[2 * i];
      ns += (double)h[2 * i + 1];
    }
    if (cyc <= 0 || ns <= 0) {
      rc = GEO_ERR_CUDA;
    } else {
      *rate = (double)kProbeThreads * kProbeIters * kProbeAcc * nsm / cyc;
      *mhz = cyc / ns * 1e3;
    }
  }
  delete[] h;
  cudaFreeAsync(rec, st);
  cudaFreeAsync(sink, st);
  return rc;
}

}  // namespace
}  // namespace geo

extern "C" GEO_API int geo_probe_minmax_rate(int form, double *lane_ops_per_clock, double *clock_mhz,
                                             void *stream) {
  using namespace geo;
  if (form < 0 || form > 3 || !lane_ops_per_clock || !clock_mhz) return GEO_ERR_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
    return GEO_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (form) {
    case 0: return run_probe<0>(nsm, st, lane_ops_per_clock, clock_mhz);
    case 1: return run_probe<1>(nsm, st, lane_ops_per_clock, clock_mhz);
    case 2: return run_probe<2>(nsm, st, lane_ops_per_clock, clock_mhz);
    default: return run_probe<3>(nsm, st, lane_ops_per_clock, clock_mhz);
  }
}
