// float64 chains, windows and reconstructions through an order-preserving
// rank transform.
//
// A geodesic step only selects among its input values (Eq. 3: extremes of
// the marker's neighbourhood and of the mask), so replacing every value by
// its rank among the distinct values of marker and mask - an order
// isomorphism - and mapping the result back gives exactly the same image.
// Each rank r goes into the chain as a rank code, the float32 whose bit
// pattern is (r + 2^16) << 7: positive, normal and finite for every r below
// kMaxRankCodes (about 2^24), ordered as the ranks, with 7 low bits that are
// always zero. The chain runs in the float32 register kernel (three-input
// max.f32 at the full 32-bit rate) instead of on int64 keys (max.s64
// emulated at about a fifth of that rate), and its passes can hand over in
// 32-bit words that carry a pass tag in those 7 bits (GEO_R32).
//
//   keys    order-preserving 64-bit keys of marker and mask (the int64 key of
//           the float64 path with the sign bit flipped, so that unsigned order
//           is numeric order; -0.0 sorts below +0.0, as there), and in the
//           same pass the global histograms of all eight 8-bit digits
//   sort    least-significant-digit radix sort of (key, position), 8 passes
//           of one kernel each (the first takes each key's position from its
//           index): a block takes the next tile by ticket, ranks its keys by
//           digit in position order (warps group equal digits by one
//           shared-memory bit per lane), publishes its digit counts and
//           finds the counts of the tiles before it by decoupled look-back
//           (bounded waits), orders the tile by digit in shared memory and
//           writes each digit's run where the global histogram (scanned by
//           every block) and the look-back put it
//   unique  one scan of the flags "key differs from its predecessor": the
//           rank of every sorted key; the distinct keys compacted and every
//           rank written back to its pixel's position
//   chain   float32 chain / window / reconstruction on the rank codes
//   unmap   out = the distinct key at the result's rank, as float64
#include <cstdlib>
#include <cstring>

#include "geo_common.cuh"
#include "geo_tile.cuh"

namespace geo {
namespace {

constexpr int kOsThreads = 256, kOsWarps = kOsThreads / 32;
constexpr int kOsTile = 2048, kOsWarpKeys = kOsTile / kOsWarps;  // keys per tile, per warp
constexpr int kDigits = 256, kPasses = 8;
constexpr int kScanThreads = 1024, kScanItems = 4, kScanTile = kScanThreads * kScanItems;
// look-back word of one tile and digit: bits 31..30 0 = not yet published,
// 1 = the tile's own count, 2 = inclusive count of all tiles up to it;
// bits 29..0 the count (at most 2^25 keys)
constexpr uint32_t kLbAgg = 1u << 30, kLbPre = 2u << 30, kLbCount = (1u << 30) - 1u;

__device__ __forceinline__ uint64_t dkey(double d) {
  const long long b = __double_as_longlong(d);
  const long long k = b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
  return (uint64_t)k ^ 0x8000000000000000ULL;
}
__device__ __forceinline__ double kdouble(uint64_t u) {
  const long long k = (long long)(u ^ 0x8000000000000000ULL);
  return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffLL));
}

// keys[0 .. H*W) = marker, keys[H*W .. 2 H*W) = mask (when given), and
// hist[p * 256 + d] += the keys whose digit p (bits 8p .. 8p + 7) is d. The
// high digits of real data take few values (sign and exponent), so the lanes
// of a warp whose digit equals lane 0's add to it with one atomic: one
// shared-memory address hit by all 32 lanes would serialise. (The kernel
// is bound by its shared-memory atomics: 8 per key. Fewer blocks with 8 keys
// a thread in flight took 51 us at 2M keys against 35 us for a block per 256
// keys.)
__global__ void __launch_bounds__(256) rk_keys(const double *__restrict__ a, const double *__restrict__ b, int64_t H,
                                               int64_t W, int64_t pitch, uint64_t *__restrict__ keys,
                                               uint32_t *__restrict__ hist) {
  __shared__ uint32_t h[kPasses * kDigits];
  for (int i = threadIdx.x; i < kPasses * kDigits; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int64_t npx = H * W, n = b ? 2 * npx : npx;
  const int lane = threadIdx.x & 31;
  // the loop is uniform per block, so every lane takes part in the votes
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < n; i0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = i0 + threadIdx.x;
    const bool valid = i < n;
    uint64_t k = 0;
    if (valid) {
      const int64_t j = i < npx ? i : i - npx;
      const int64_t o = pitch == W ? j : (j / W) * pitch + j % W;
      k = dkey(i < npx ? a[o] : b[o]);
      keys[i] = k;
    }
#pragma unroll
    for (int p = 0; p < kPasses; ++p) {
      const unsigned d = valid ? (unsigned)((k >> (8 * p)) & 255u) : 256u;
      const unsigned lead = __shfl_sync(0xffffffffu, d, 0);
      const unsigned same = __ballot_sync(0xffffffffu, d == lead);
      if (valid) {
        if (d != lead) atomicAdd(&h[p * kDigits + (int)d], 1u);
        else if (lane == 0) atomicAdd(&h[p * kDigits + (int)d], (unsigned)__popc(same));
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kPasses * kDigits; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
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

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One pass of the radix sort of (key, pos) on the digit at `shift` (pin ==
// nullptr: the positions are the indices, in the first pass).
// A block takes tile t by ticket (so every tile before t belongs to a block
// that is already running: the look-back waits always end), and warp w owns
// keys [w * 256, (w + 1) * 256) of the tile, 8 per lane held in registers
// and walked in rounds of 32 in position order (warp_digit_peers groups the
// lanes of equal digits): first counting each digit, then placing each key in
// shared memory at the tile's start of its digit + the counts of earlier
// warps + the keys of its digit seen earlier in the warp + the lanes below
// it in the round with the same digit (a stable local sort by digit). The
// tile's digit counts are published before that placement and the tiles
// before it are looked up after it (decoupled look-back over per-tile,
// per-digit words: a tile's own count, or the inclusive count once the tile
// knows it; each lane reads kLbWindow predecessors at once), so that the
// counts of most earlier tiles are there when needed. Digit d's keys of the
// tile then go, contiguously, to the digit's first output position (the
// exclusive prefix of the pass's global histogram, which every block scans
// for itself) + the sum found. A look-back wait that expires (limit_ns)
// records GEO_ERR_TIMEOUT and the block writes nothing.
// 8 predecessors a read. Measured transform time at 2M keys by window: 1:
// 0.44 ms, 2: 0.42, 4: 0.40, 8: 0.40, 16: 0.48, 32: 0.63 (the wider reads of
// a spinning look-back take issue slots that the other blocks on the SM
// need; pausing between them changed nothing).
constexpr int kLbWindow = 8;
constexpr int kOsRounds = kOsWarpKeys / 32;  // keys per lane

// The lanes of the warp whose digit equals this lane's (d < 256; a lane with
// d >= 256 has no peers): each lane sets its bit in the warp's word of its
// digit, reads the word back, and the lowest lane of each group clears it
// for the next round. (__match_any_sync gives the same masks, but measured
// about 1000 SM clocks a call with some 30 distinct digits among 32 lanes.)
__device__ __forceinline__ unsigned warp_digit_peers(uint32_t *wm, unsigned d, int lane) {
  const unsigned me = 1u << lane;
  if (d < 256u) atomicOr(&wm[d], me);
  __syncwarp();
  const unsigned peers = d < 256u ? wm[d] : me;
  __syncwarp();
  if (d < 256u && (peers & (me - 1u)) == 0) wm[d] = 0;
  __syncwarp();
  return peers;
}
__global__ void __launch_bounds__(kOsThreads, 4) rk_onesweep(const uint64_t *__restrict__ kin,
                                                          const uint32_t *__restrict__ pin, uint64_t *__restrict__ kout,
                                                          uint32_t *__restrict__ pout, int64_t n, int shift,
                                                          const uint32_t *__restrict__ hist, uint32_t *lookback,
                                                          uint32_t *ticket, int *status,
                                                          unsigned long long limit_ns) {
  extern __shared__ __align__(16) char os_dyn[];
  uint64_t *sk = reinterpret_cast<uint64_t *>(os_dyn);               // the tile's keys, by digit
  uint32_t *sp = reinterpret_cast<uint32_t *>(os_dyn + 8 * kOsTile);  // and their positions
  __shared__ uint32_t cnt[kOsWarps][kDigits];
  __shared__ uint32_t wmask[kOsWarps][kDigits];  // warp_digit_peers' words
  __shared__ uint32_t dend[kDigits], tcnt[kDigits], gbase[kDigits], doff[kDigits];
  __shared__ int tile_s, fail_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    tile_s = (int)atomicAdd(ticket, 1u);
    fail_s = 0;
  }
  for (int i = threadIdx.x; i < kOsWarps * kDigits; i += kOsThreads) {
    (&cnt[0][0])[i] = 0;
    (&wmask[0][0])[i] = 0;
  }
  __syncthreads();
  const int tile = tile_s;
  const int64_t wbase = (int64_t)tile * kOsTile + (int64_t)warp * kOsWarpKeys;
  const unsigned lt = (1u << lane) - 1u;
  // the lane's keys of every round, all loads in flight together
  uint64_t k[kOsRounds];
  uint32_t pk[kOsRounds];
#pragma unroll
  for (int r = 0; r < kOsRounds; ++r) {
    const int64_t idx = wbase + 32 * r + lane;
    k[r] = idx < n ? kin[idx] : 0ull;
    pk[r] = idx < n ? (pin ? pin[idx] : (uint32_t)idx) : 0u;
  }
#pragma unroll
  for (int r = 0; r < kOsRounds; ++r) {
    const int64_t idx = wbase + 32 * r + lane;
    const unsigned d = idx < n ? (unsigned)((k[r] >> shift) & 255u) : 256u;  // past the end: no peers
    const unsigned peers = warp_digit_peers(wmask[warp], d, lane);
    if (d < 256u && (peers & lt) == 0) cnt[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    const int d = threadIdx.x;  // one thread per digit
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < kOsWarps; ++w) {
      const uint32_t x = cnt[w][d];
      cnt[w][d] = c;  // the warp's start within the digit's keys of this tile
      c += x;
    }
    tcnt[d] = c;
    dend[d] = c;
    st_relaxed_u32(lookback + (int64_t)tile * kDigits + d, (tile == 0 ? kLbPre : kLbAgg) | c);
    doff[d] = hist[d];
  }
  __syncthreads();
  // inclusive scans over the digits: dend[d], the tile's keys of digits <= d;
  // doff[d], all keys of digits <= d (made exclusive below)
  for (int o = 1; o < kDigits; o <<= 1) {
    const uint32_t t = threadIdx.x >= (unsigned)o ? dend[threadIdx.x - o] : 0u;
    const uint32_t u = threadIdx.x >= (unsigned)o ? doff[threadIdx.x - o] : 0u;
    __syncthreads();
    dend[threadIdx.x] += t;
    doff[threadIdx.x] += u;
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < kOsRounds; ++r) {
    const int64_t idx = wbase + 32 * r + lane;
    const bool valid = idx < n;
    const unsigned d = valid ? (unsigned)((k[r] >> shift) & 255u) : 256u;
    const unsigned peers = warp_digit_peers(wmask[warp], d, lane);
    if (valid) {
      const uint32_t at = (d == 0 ? 0u : dend[d - 1]) + cnt[warp][d] + __popc(peers & lt);
      sk[at] = k[r];
      sp[at] = pk[r];
    }
    __syncwarp();
    if (valid && (peers & lt) == 0) cnt[warp][d] += __popc(peers);
    __syncwarp();
  }
  {
    // look-back for digit d over the tiles before this one, kLbWindow at a time
    const int d = threadIdx.x;
    uint32_t before = 0;
    if (tile > 0) {
      unsigned long long t0 = 0;
      unsigned spins = 0;
      int j = tile - 1;
      bool done = false;
      while (!done) {
        uint32_t wv[kLbWindow];
#pragma unroll
        for (int q = 0; q < kLbWindow; ++q)
          wv[q] = (j - q >= 0) ? ld_relaxed_u32(lookback + (int64_t)(j - q) * kDigits + d) : kLbPre;
        // nearest first: add counts until an inclusive one; stop at the first unpublished word
        int q = 0;
        for (; q < kLbWindow && j - q >= 0; ++q) {
          const uint32_t w = wv[q];
          if ((w >> 30) == 0u) break;
          before += w & kLbCount;
          if ((w >> 30) == 2u) {
            done = true;
            break;
          }
        }
        if (done) break;
        if (q == 0) {  // the nearest word not published yet: wait (bounded)
          if (spins == 0) t0 = globaltimer_ns();
          if ((++spins & 63u) == 0 && globaltimer_ns() - t0 > limit_ns) {
            fail_s = 1;
            break;
          }
          continue;
        }
        j -= q;
        if (j < 0) break;  // cannot happen: tile 0's word is inclusive
      }
      st_relaxed_u32(lookback + (int64_t)tile * kDigits + d, kLbPre | (before + tcnt[d]));
    }
    gbase[d] = doff[d] - hist[d] + before;  // exclusive: the first output position of digit d
  }
  __syncthreads();
  if (fail_s) {
    if (threadIdx.x == 0) record_status(status, GEO_ERR_TIMEOUT);
    return;
  }
  const int64_t t0 = (int64_t)tile * kOsTile;
  const int tn = (int)((n - t0) < kOsTile ? (n - t0) : kOsTile);
  for (int i = threadIdx.x; i < tn; i += kOsThreads) {
    const uint64_t k = sk[i];
    const unsigned d = (unsigned)((k >> shift) & 255u);
    const int64_t o = (int64_t)gbase[d] + (i - (int64_t)(d == 0 ? 0u : dend[d - 1]));
    if (o >= 0 && o < n) {
      kout[o] = k;
      pout[o] = sp[i];
    }
  }
}

// The run-start flags of the sorted keys (1 where a key differs from its
// predecessor), scanned per block of kScanTile: v = the exclusive scan within
// the block, sums = the block totals (scanned by rk_scan_small; rk_finish
// adds them back).
__global__ void __launch_bounds__(kScanThreads) rk_scan_blocks(const uint64_t *__restrict__ s, uint32_t *__restrict__ v,
                                                               int64_t n, uint32_t *__restrict__ sums) {
  static_assert(kScanThreads == 32 * 32, "one warp scans the warp totals");
  __shared__ uint32_t wsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * kScanTile;
  uint32_t loc[kScanItems], sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = c0 + (int64_t)threadIdx.x * kScanItems + i;
    loc[i] = idx < n ? ((idx == 0 || s[idx] != s[idx - 1]) ? 1u : 0u) : 0u;
    sum += loc[i];
  }
  // inclusive scan of the thread sums: within each warp by shuffles, then
  // of the 32 warp totals by warp 0
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    wsum[lane] = t;
  }
  __syncthreads();
  uint32_t run = (warp ? wsum[warp - 1] : 0u) + x - sum;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = c0 + (int64_t)threadIdx.x * kScanItems + i;
    if (idx < n) v[idx] = run;
    run += loc[i];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = wsum[31];
}

// After the scan of the run-start flags (exclusive: the block's scan plus
// the scanned block total): the rank of sorted key i among the distinct keys
// is scan[i] + flag[i] - 1. The run starts go to uniq[rank], and every rank's
// code to the key's position: codes[pos[i]] (marker then mask, as the keys
// were laid out).
__global__ void rk_finish(const uint64_t *__restrict__ s, const uint32_t *__restrict__ pos,
                          const uint32_t *__restrict__ flags_scan, const uint32_t *__restrict__ block_sums, int64_t n,
                          uint64_t *__restrict__ uniq, float *__restrict__ codes) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = s[i];
    const bool start = (i == 0 || k != s[i - 1]);
    const uint32_t r = flags_scan[i] + block_sums[i / kScanTile] + (start ? 1u : 0u) - 1u;
    if (start) uniq[r] = k;
    codes[pos[i]] = __uint_as_float((r + kRankCodeBase) << 7);
  }
}

__global__ void rk_unmap(const float *__restrict__ r, int64_t H, int64_t W, const uint64_t *__restrict__ uniq,
                         double *__restrict__ out, int64_t pitch) {
  const int64_t n = H * W;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / W, x = i - y * W;
    out[y * pitch + x] = kdouble(uniq[(__float_as_uint(r[i]) >> 7) - kRankCodeBase]);
  }
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

int ew_grid(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

bool rank_path_applies(int64_t H, int64_t W, bool has_mask, int mode, int64_t steps) {
  const char *e = getenv("GEOMORPH_F64");
  if (e && strcmp(e, "keys") == 0) return false;
  const int64_t n = H * W * (has_mask ? 2 : 1);
  if (n > kMaxRankCodes) return false;  // every rank code must stay below +inf
  if (e && strcmp(e, "ranks") == 0) return true;
  // At 1024^2 a call on the rank codes costs about 0.39 ms + 0.62 us a step
  // (radix sort, ranks, map back, the tagged float32 chain), one on int64
  // keys about 3.2-3.8 us a step, so the ranks pay from about 140 steps on.
  // Reconstruction takes its chain length from the image's longer side.
  // Small images stay on the keys (the launches of the transform dominate
  // there).
  const int64_t est = mode == MODE_REC ? (H > W ? H : W) : steps;
  return est >= 160 && H * W >= ((int64_t)1 << 16);
}

int run_chain_ranked(const double *marker, const double *mask, double *out, int64_t H, int64_t W, int64_t pitch,
                     int conn, int op, int mode, int64_t steps, int64_t *steps_out, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t npx = H * W, n = npx * (mask ? 2 : 1);
  const int ntiles = (int)((n + kOsTile - 1) / kOsTile);
  const int64_t nsb = (n + kScanTile - 1) / kScanTile;
  // scratch: [keys A][keys B][pos A][pos B][uniq][flag scan][digit histograms][scan block sums][U]
  //          [tickets][look-back words, per pass][ranks: marker, mask][ranks out]
  const size_t kb = up256((size_t)n * 8), pb = up256((size_t)n * 4), fb = up256((size_t)n * 4);
  const size_t hb = up256((size_t)kPasses * kDigits * 4), sb = up256((size_t)(nsb > 0 ? nsb : 1) * 4);
  const size_t lbb = up256((size_t)kPasses * ntiles * kDigits * 4), rb = up256((size_t)npx * 4);
  const size_t total = 3 * kb + 2 * pb + fb + hb + sb + 256 + 256 + lbb + 3 * rb;
  void *scratch = nullptr;
  int rc = pool_alloc(&scratch, total, s);
  if (rc != GEO_OK) return rc;
  int *status = nullptr;
  if (device_status_word(&status) != GEO_OK) {
    pool_free(scratch, s);
    return GEO_ERR_CUDA;
  }
  char *p = (char *)scratch;
  uint64_t *ka = (uint64_t *)p, *kbuf = (uint64_t *)(p + kb), *uniq = (uint64_t *)(p + 2 * kb);
  p += 3 * kb;
  uint32_t *pa = (uint32_t *)p, *pbuf = (uint32_t *)(p + pb);
  p += 2 * pb;
  uint32_t *flags = (uint32_t *)p;
  p += fb;
  uint32_t *hist = (uint32_t *)p;  // digit histograms of the 8 passes
  p += hb;
  uint32_t *bsums = (uint32_t *)p;
  p += sb;
  uint32_t *U = (uint32_t *)p;
  p += 256;
  uint32_t *tickets = (uint32_t *)p;
  uint32_t *lookback = (uint32_t *)(p + 256);
  p += 256 + lbb;
  float *rm = (float *)p, *rk = (float *)(p + (mask ? (size_t)npx * 4 : 0)), *ro = (float *)(p + 2 * rb);
  // (marker and mask ranks contiguous: ranks[pos] with pos < npx the marker's)

  if (cudaMemsetAsync(hist, 0, hb, s) != cudaSuccess ||
      cudaMemsetAsync(tickets, 0, 256 + lbb, s) != cudaSuccess)
    rc = GEO_ERR_CUDA;
  // the one-sweep kernel's tile (keys and positions) takes 48 KB of dynamic
  // shared memory next to its static counts
  const int os_smem = kOsTile * (8 + 4);
  if (cudaFuncSetAttribute(rk_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize, os_smem) != cudaSuccess ||
      cudaFuncSetAttribute(rk_onesweep, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    rc = GEO_ERR_CUDA;
  const bool fault = host_fault() == FAULT_TIMEOUT;
  const unsigned long long limit = fault ? kFaultWaitNs : kWaitLimitNs;
  if (rc == GEO_OK) {
    rk_keys<<<ew_grid(n), 256, 0, s>>>(marker, mask, H, W, pitch, ka, hist);
    uint64_t *ks = ka, *kd = kbuf;
    uint32_t *ps = nullptr, *pd = pa;  // the first pass takes the positions from the indices
    for (int pass = 0; pass < kPasses; ++pass) {
      rk_onesweep<<<ntiles, kOsThreads, os_smem, s>>>(ks, ps, kd, pd, n, 8 * pass, hist + pass * kDigits,
                                                      lookback + (size_t)pass * ntiles * kDigits, tickets + pass,
                                                      status, limit);
      uint64_t *t = ks;
      ks = kd;
      kd = t;
      ps = pd;
      pd = (pd == pa) ? pbuf : pa;
    }
    // 8 passes: the sorted keys are back in ka, their positions in pbuf (ks / ps)
    rk_scan_blocks<<<(unsigned)nsb, kScanThreads, 0, s>>>(ks, flags, n, bsums);
    rk_scan_small<<<1, kScanThreads, 0, s>>>(bsums, nsb, U);
    rk_finish<<<ew_grid(n), 256, 0, s>>>(ks, ps, flags, bsums, n, uniq, rm);
    if (cudaGetLastError() != cudaSuccess) rc = GEO_ERR_CUDA;
  }
  if (rc == GEO_OK)
    rc = run_chain_any(GEO_R32, rm, mask ? rk : nullptr, ro, H, W, W, conn, op, mode, steps, steps_out, stream, 1);
  if (rc == GEO_OK) {
    rk_unmap<<<ew_grid(npx), 256, 0, s>>>(ro, H, W, uniq, out, pitch);
    if (cudaGetLastError() != cudaSuccess) rc = GEO_ERR_CUDA;
  }
  if (pool_free(scratch, s) != GEO_OK && rc == GEO_OK) rc = GEO_ERR_CUDA;
  return rc;
}

}  // namespace geo
