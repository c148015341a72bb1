// float64 chains, windows and reconstructions through an order-preserving
// rank transform.
//
// A geodesic step only selects among its input values (Eq. 3: extremes of
// the marker's neighbourhood and of the mask), so replacing every value by
// its rank among the distinct values of marker and mask - an order
// isomorphism - and mapping the result back gives exactly the same image.
// With at most 2^24 distinct values the ranks are exact float32 integers, and
// the chain runs in the float32 register kernel (three-input max.f32 at the
// full 32-bit rate) instead of on int64 keys (max.s64 emulated at about a
// fifth of that rate).
//
//   keys    order-preserving 64-bit keys of marker and mask (the int64 key of
//           the float64 path with the sign bit flipped, so that unsigned order
//           is numeric order; -0.0 sorts below +0.0, as there)
//   sort    least-significant-digit radix sort, 8 passes of 8 bits: per block
//           digit histogram, one scan, stable scatter (warps rank equal
//           digits with __match_any_sync, in key order)
//   unique  flags where a key differs from its predecessor, scan, compact
//   map     rank of each pixel by binary search among the distinct keys
//   chain   float32 chain / window / reconstruction on the ranks
//   unmap   out = the distinct key at the result's rank, as float64
#include <cstdlib>
#include <cstring>

#include "geo_common.cuh"

namespace geo {
namespace {

constexpr int kRsThreads = 256, kRsItems = 16, kRsTile = kRsThreads * kRsItems;  // 4096 keys per block
constexpr int kRsWarps = kRsThreads / 32, kRsWarpKeys = kRsTile / kRsWarps;      // 512 keys per warp
constexpr int kScanThreads = 1024, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint64_t dkey(double d) {
  const long long b = __double_as_longlong(d);
  const long long k = b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
  return (uint64_t)k ^ 0x8000000000000000ULL;
}
__device__ __forceinline__ double kdouble(uint64_t u) {
  const long long k = (long long)(u ^ 0x8000000000000000ULL);
  return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffLL));
}

// keys[0 .. H*W) = marker, keys[H*W .. 2 H*W) = mask (when given)
__global__ void rk_keys(const double *__restrict__ a, const double *__restrict__ b, int64_t H, int64_t W,
                        int64_t pitch, uint64_t *__restrict__ keys) {
  const int64_t n = H * W;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / W, x = i - y * W;
    keys[i] = dkey(a[y * pitch + x]);
    if (b) keys[n + i] = dkey(b[y * pitch + x]);
  }
}

// per-block histogram of one digit: hist[digit * nblocks + block]
__global__ void __launch_bounds__(kRsThreads) rk_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                                                      uint32_t *__restrict__ hist, int nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll 4
  for (int i = threadIdx.x; i < kRsTile; i += kRsThreads) {
    const int64_t idx = base + i;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of n uint32 in place, one block, in chunks of kScanTile
// (the running total carries from chunk to chunk). total (optional) gets the
// sum of all n.
__global__ void __launch_bounds__(kScanThreads) rk_scan_small(uint32_t *__restrict__ v, int64_t n,
                                                              uint32_t *total) {
  __shared__ uint32_t part[kScanThreads];
  __shared__ uint32_t carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < n; c0 += kScanTile) {
    uint32_t loc[kScanItems], sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      const int64_t idx = c0 + (int64_t)threadIdx.x * kScanItems + i;
      loc[i] = idx < n ? v[idx] : 0u;
      sum += loc[i];
    }
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {  // inclusive scan of the thread sums
      const uint32_t t = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
      __syncthreads();
      part[threadIdx.x] += t;
      __syncthreads();
    }
    uint32_t run = carry_s + part[threadIdx.x] - sum;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      const int64_t idx = c0 + (int64_t)threadIdx.x * kScanItems + i;
      if (idx < n) v[idx] = run;
      run += loc[i];
    }
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry_s += part[kScanThreads - 1];
    __syncthreads();
  }
  if (total && threadIdx.x == 0) *total = carry_s;
}

// Stable scatter of one digit. Warp w of a block owns keys [w * 512, (w + 1)
// * 512) of the block's tile and walks them in rounds of 32 in key order:
// first counting each digit, then placing each key at the block's offset of
// its digit + the counts of earlier warps + the keys of its digit seen
// earlier in the warp + the lanes below it in the round with the same digit.
__global__ void __launch_bounds__(kRsThreads) rk_scatter(const uint64_t *__restrict__ in, uint64_t *__restrict__ out,
                                                         int64_t n, int shift, const uint32_t *__restrict__ hist,
                                                         int nblocks) {
  __shared__ uint32_t cnt[kRsWarps][256];
  __shared__ uint32_t base_s[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&cnt[0][0])[i] = 0;
  base_s[threadIdx.x] = hist[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  __syncthreads();
  const int64_t wbase = (int64_t)blockIdx.x * kRsTile + (int64_t)warp * kRsWarpKeys;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kRsWarpKeys; r += 32) {
    const int64_t idx = wbase + r + lane;
    const unsigned d = idx < n ? (unsigned)((in[idx] >> shift) & 255u) : 256u + lane;  // past the end: no peers
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (d < 256u && (peers & lt) == 0) cnt[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive prefix over the warps, then the block's offset
  {
    const int d = threadIdx.x;  // 256 threads, one per digit
    uint32_t run = base_s[d];
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) {
      const uint32_t c = cnt[w][d];
      cnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int r = 0; r < kRsWarpKeys; r += 32) {
    const int64_t idx = wbase + r + lane;
    const bool valid = idx < n;
    const uint64_t k = valid ? in[idx] : 0ull;
    const unsigned d = valid ? (unsigned)((k >> shift) & 255u) : 256u + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (valid) out[cnt[warp][d] + __popc(peers & lt)] = k;
    __syncwarp();
    if (valid && (peers & lt) == 0) cnt[warp][d] += __popc(peers);
    __syncwarp();
  }
}

// flags[i] = 1 where sorted[i] starts a run of equal keys
__global__ void rk_flags(const uint64_t *__restrict__ s, int64_t n, uint32_t *__restrict__ f) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    f[i] = (i == 0 || s[i] != s[i - 1]) ? 1u : 0u;
}

// Exclusive scan of large arrays: per-block scans, block sums scanned by
// rk_scan_small, then added back.
__global__ void __launch_bounds__(kScanThreads) rk_scan_blocks(uint32_t *__restrict__ v, int64_t n,
                                                               uint32_t *__restrict__ sums) {
  __shared__ uint32_t part[kScanThreads];
  const int64_t c0 = (int64_t)blockIdx.x * kScanTile;
  uint32_t loc[kScanItems], sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = c0 + (int64_t)threadIdx.x * kScanItems + i;
    loc[i] = idx < n ? v[idx] : 0u;
    sum += loc[i];
  }
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {
    const uint32_t t = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += t;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - sum;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = c0 + (int64_t)threadIdx.x * kScanItems + i;
    if (idx < n) v[idx] = run;
    run += loc[i];
  }
  if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = part[kScanThreads - 1];
}

__global__ void rk_scan_add(uint32_t *__restrict__ v, int64_t n, const uint32_t *__restrict__ sums) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx < n) v[idx] += sums[idx / kScanTile];
}

// compact the run starts: uniq[scan[i]] = sorted[i] where flags[i]
__global__ void rk_compact(const uint64_t *__restrict__ s, const uint32_t *__restrict__ flags_scan, int64_t n,
                           uint64_t *__restrict__ uniq) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (i == 0 || s[i] != s[i - 1]) uniq[flags_scan[i]] = s[i];
  }
}

// Bucket table of the distinct keys by their top kPrefixBits: the keys with
// prefix p are uniq[start[p] .. end[p]). Only prefixes that occur are
// written, and only those are read (every looked-up key is present).
constexpr int kPrefixBits = 20;
__device__ __forceinline__ uint32_t key_prefix(uint64_t k) { return (uint32_t)(k >> (64 - kPrefixBits)); }

__global__ void rk_buckets(const uint64_t *__restrict__ uniq, const uint32_t *__restrict__ U, int64_t n,
                           uint32_t *__restrict__ start, uint32_t *__restrict__ end) {
  const int64_t u = *U;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n && i < u;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t p = key_prefix(uniq[i]);
    if (i == 0 || key_prefix(uniq[i - 1]) != p) start[p] = (uint32_t)i;
    if (i == u - 1 || key_prefix(uniq[i + 1]) != p) end[p] = (uint32_t)(i + 1);
  }
}

// ranks (as float32) of an image's values among the distinct keys: binary
// search inside the key's prefix bucket
__global__ void rk_map(const double *__restrict__ a, int64_t H, int64_t W, int64_t pitch,
                       const uint64_t *__restrict__ uniq, const uint32_t *__restrict__ start,
                       const uint32_t *__restrict__ end, float *__restrict__ r) {
  const int64_t n = H * W;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / W, x = i - y * W;
    const uint64_t k = dkey(a[y * pitch + x]);
    const uint32_t p = key_prefix(k);
    uint32_t lo = start[p], hi = end[p];  // first index with uniq >= k (the key is present)
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (uniq[mid] < k) lo = mid + 1;
      else hi = mid;
    }
    r[i] = (float)lo;
  }
}

__global__ void rk_unmap(const float *__restrict__ r, int64_t H, int64_t W, const uint64_t *__restrict__ uniq,
                         double *__restrict__ out, int64_t pitch) {
  const int64_t n = H * W;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / W, x = i - y * W;
    out[y * pitch + x] = kdouble(uniq[(uint32_t)r[i]]);
  }
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

int ew_grid(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

// device-wide exclusive scan of n uint32; block_sums holds one entry per
// kScanTile elements (scanned by one block in chunks)
int scan_u32(uint32_t *v, int64_t n, uint32_t *block_sums, uint32_t *total, cudaStream_t s) {
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  rk_scan_blocks<<<(unsigned)nb, kScanThreads, 0, s>>>(v, n, block_sums);
  rk_scan_small<<<1, kScanThreads, 0, s>>>(block_sums, nb, total);
  rk_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, n, block_sums);
  return cudaGetLastError() == cudaSuccess ? GEO_OK : GEO_ERR_CUDA;
}

}  // namespace

bool rank_path_applies(int64_t H, int64_t W, bool has_mask, int mode, int64_t steps) {
  const char *e = getenv("GEOMORPH_F64");
  if (e && strcmp(e, "keys") == 0) return false;
  const int64_t n = H * W * (has_mask ? 2 : 1);
  if (n > ((int64_t)1 << 24)) return false;  // ranks must stay exact float32 integers
  if (e && strcmp(e, "ranks") == 0) return true;
  // The transform costs about 0.5 ms at 1024^2 (radix sort, ranks, map
  // back), about 200 int64-key steps there; reconstruction takes its chain
  // length from the image's longer side. Small images stay on the keys (the
  // launches of the transform dominate there).
  const int64_t est = mode == MODE_REC ? (H > W ? H : W) : steps;
  return est >= 256 && H * W >= ((int64_t)1 << 16);
}

int run_chain_ranked(const double *marker, const double *mask, double *out, int64_t H, int64_t W, int64_t pitch,
                     int conn, int op, int mode, int64_t steps, int64_t *steps_out, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t npx = H * W, n = npx * (mask ? 2 : 1);
  const int nblocks = (int)((n + kRsTile - 1) / kRsTile);
  const int64_t nsb = (n + kScanTile - 1) / kScanTile;
  // scratch: [keys A][keys B][uniq][flags/scan][hist][scan block sums][U][ranks: marker, mask, out]
  //          [bucket start][bucket end]
  const size_t kb = up256((size_t)n * 8), fb = up256((size_t)n * 4), hb = up256((size_t)256 * nblocks * 4);
  const size_t sb = up256((size_t)(nsb > 0 ? nsb : 1) * 4), rb = up256((size_t)npx * 4);
  const size_t tb = (size_t)4 << kPrefixBits;
  const size_t total = 3 * kb + fb + hb + sb + 256 + 3 * rb + 2 * tb;
  void *scratch = nullptr;
  int rc = pool_alloc(&scratch, total, s);
  if (rc != GEO_OK) return rc;
  char *p = (char *)scratch;
  uint64_t *ka = (uint64_t *)p, *kbuf = (uint64_t *)(p + kb), *uniq = (uint64_t *)(p + 2 * kb);
  uint32_t *flags = (uint32_t *)(p + 3 * kb), *hist = (uint32_t *)(p + 3 * kb + fb);
  uint32_t *bsums = (uint32_t *)(p + 3 * kb + fb + hb), *U = (uint32_t *)(p + 3 * kb + fb + hb + sb);
  float *rm = (float *)(p + 3 * kb + fb + hb + sb + 256), *rk = (float *)((char *)rm + rb);
  float *ro = (float *)((char *)rm + 2 * rb);
  uint32_t *bstart = (uint32_t *)((char *)rm + 3 * rb), *bend = (uint32_t *)((char *)rm + 3 * rb + tb);

  rk_keys<<<ew_grid(npx), 256, 0, s>>>(marker, mask, H, W, pitch, ka);
  uint64_t *src = ka, *dst = kbuf;
  for (int shift = 0; shift < 64; shift += 8) {
    rk_hist<<<nblocks, kRsThreads, 0, s>>>(src, n, shift, hist, nblocks);
    if (scan_u32(hist, (int64_t)256 * nblocks, bsums, nullptr, s) != GEO_OK) rc = GEO_ERR_CUDA;
    rk_scatter<<<nblocks, kRsThreads, 0, s>>>(src, dst, n, shift, hist, nblocks);
    uint64_t *t = src;
    src = dst;
    dst = t;
  }
  // 8 passes: the sorted keys are back in ka (src)
  rk_flags<<<ew_grid(n), 256, 0, s>>>(src, n, flags);
  if (cudaGetLastError() != cudaSuccess) rc = GEO_ERR_CUDA;
  if (rc == GEO_OK) rc = scan_u32(flags, n, bsums, U, s);
  if (rc == GEO_OK) {
    rk_compact<<<ew_grid(n), 256, 0, s>>>(src, flags, n, uniq);
    rk_buckets<<<ew_grid(n), 256, 0, s>>>(uniq, U, n, bstart, bend);
    rk_map<<<ew_grid(npx), 256, 0, s>>>(marker, H, W, pitch, uniq, bstart, bend, rm);
    if (mask) rk_map<<<ew_grid(npx), 256, 0, s>>>(mask, H, W, pitch, uniq, bstart, bend, rk);
    if (cudaGetLastError() != cudaSuccess) rc = GEO_ERR_CUDA;
  }
  if (rc == GEO_OK)
    rc = run_chain_any(GEO_F32, rm, mask ? rk : nullptr, ro, H, W, W, conn, op, mode, steps, steps_out, stream, 1);
  if (rc == GEO_OK) {
    rk_unmap<<<ew_grid(npx), 256, 0, s>>>(ro, H, W, uniq, out, pitch);
    if (cudaGetLastError() != cudaSuccess) rc = GEO_ERR_CUDA;
  }
  if (pool_free(scratch, s) != GEO_OK && rc == GEO_OK) rc = GEO_ERR_CUDA;
  return rc;
}

}  // namespace geo
