// Openings, closings, granulometry with its pattern spectrum, and alternating
// sequential filters (Section 2, Eq. 16-20), on the register engine's
// unmasked 3x3 chains (s elementary steps for a (2s+1)^2 square).
//
// * gamma_s(f) = delta_s(eps_s(f)), phi_s(f) = eps_s(delta_s(f)) and
//   ASF_s = phi_s gamma_s ... phi_1 gamma_1 are programs of runs of one
//   operation (prog_kernel below), each one persistent launch. ASF_s is the
//   sequence of elementary steps E1 D1 D1 E1 E2 D2 D2 E2 ... Es Ds Ds Es
//   (E = eps_1, D = delta_1, counts as written); runs of the same operation
//   are merged (E1, D2, E3, D4, ..., D2s, Es): the same steps in the same
//   order.
// * G_s = sum of gamma_s(f) for s = 0..smax: eps_s(f) is kept and eroded one
//   more step for each s (eps_s = eps_1 eps_{s-1} by Eq. 4's nesting), the
//   dilation of s steps goes to a second buffer, and a two-stage reduction
//   sums it in double (fixed partition and order: deterministic; exact for
//   uint8 images). PS_s = G_s - G_{s+1}.
#include <cstring>
#include <vector>

#include "geo_rr.cuh"

namespace geo {
namespace {

// ---------------------------------------------------------------------------
// Programs of unmasked 8-connected runs (erode or dilate, n elementary steps
// each) in one persistent launch of the register engine: the passes of all
// runs are numbered in order and synchronised point to point through the
// per-tile epochs exactly as one chain's passes are; each pass runs the
// policy of its run, with the virtual mask and the exchange buffer's
// identity rows of that operation.
// ---------------------------------------------------------------------------

constexpr int kMaxRuns = 48;

struct Program {
  int nruns;
  int total_passes;
  int op[kMaxRuns];
  int npasses[kMaxRuns];
  int64_t steps[kMaxRuns];
};

// One pass of one tile. TAG: the uint8 form whose passes hand over in the
// tagged planes of TileLaunch::tagged (as the chains of rr_kernel do): tin
// (else the plain src) is read waiting for tag `want`, tout (else the plain
// dst) is written with tag want + 1.
template <class P, bool TAG>
__device__ __forceinline__ bool prog_tile(const TileLaunch &L, const Plane &src, const Plane &dst, bool src_cg,
                                          const unsigned long long *tin, unsigned long long *tout, unsigned want,
                                          int64_t ty0, int64_t tx0, int S, typename P::Wd *xb0, int xb_stride,
                                          uint64_t *bar, int &parity, int lane, int warp,
                                          typename P::Wd (&w)[P::RW][P::CW], typename P::Wd (&m)[P::RW][P::CW]) {
  using R = RR<P>;
  const int K = L.K;
  const int64_t gy0 = ty0 - K + warp * R::PH, gx = tx0 - K + lane * R::CW;
  bool ok = true, loaded = false;
  if constexpr (TAG) {
    if (tin) {
      ok = R::load_tagged(tin, L.tpitch, L.H, L.W, gy0, gx, L.fault ? want + (1u << 28) : want, L.wait_ns, w);
      loaded = true;
    }
  }
  if (!loaded) R::load_words(src, L.H, L.W, gy0, gx, src_cg, false, w);
  R::load_words(src, L.H, L.W, gy0, gx, false, true, m);  // the virtual mask of this operation
  // tagged hand-over: no fence between the pass's loads and its stores, by
  // the same write-after-read argument as in rr_kernel (every store of a
  // pass depends on that pass's tag checks)
  for (int j = 0; j < S; ++j) {
    ok &= R::template step<8>(w, m, xb0 + (size_t)parity * xb_stride, bar, parity, lane, warp);
    parity ^= 1;
  }
  bool stored = false;
  if constexpr (TAG) {
    if (tout) {
      R::store_tagged(w, tout, L.tpitch, L.H, L.W, ty0, tx0, K, L.TH, L.TW, want + 1, lane, warp);
      stored = true;
    }
  }
  if (!stored) R::store(w, dst, src, false, L.H, L.W, ty0, tx0, K, L.TH, L.TW, lane, warp);
  return ok;
}

template <template <int> class RP, bool TAG = false>
__global__ void __launch_bounds__(RP<DILATE>::NW * 32, 1) prog_kernel(const TileLaunch L, const Program G) {
  using PD = RP<DILATE>;
  using PE = RP<ERODE>;
  using Wd = typename PD::Wd;
  constexpr int CW = PD::CW, RW = PD::RW, NW = PD::NW, RWID = 32 * CW;
  extern __shared__ __align__(16) char rr_dyn[];
  Wd(*xbuf)[NW + 2][2][RWID] = reinterpret_cast<Wd(*)[NW + 2][2][RWID]>(rr_dyn);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntiles = L.tiles_x * L.tiles_y;
  __shared__ __align__(8) uint64_t xbar;
  if (threadIdx.x == 0) mbar_init(&xbar, NW * 32);
  Wd w[RW][CW], m[RW][CW];
  int parity = 0, cur_op = -1, p = 0;
  for (int r = 0; r < G.nruns; ++r) {
    const int op = G.op[r];
    if (op != cur_op) {
      // the rows above warp 0 and below warp NW-1 hold this operation's identity
      __syncthreads();
      const Wd id = op == DILATE ? PD::identw() : PE::identw();
      for (int i = threadIdx.x; i < 2 * 2 * RWID; i += NW * 32) {
        const int par = i / (2 * RWID), rest = i % (2 * RWID);
        (&xbuf[par][0][0][0])[rest] = id;
        (&xbuf[par][NW + 1][0][0])[rest] = id;
      }
      __syncthreads();
      cur_op = op;
    }
    const int np = G.npasses[r];
    const int64_t base = np > 0 ? G.steps[r] / np : 0, extra = np > 0 ? G.steps[r] % np : 0;
    for (int q = 0; q < np; ++q, ++p) {
      const int S = (int)(base + (q < extra ? 1 : 0));
      const bool to_out = ((G.total_passes - 1 - p) & 1) == 0;
      const Plane dst = to_out ? L.out : L.scratch;
      const Plane src = p == 0 ? L.marker : (to_out ? L.scratch : L.out);
      const bool src_cg = p > 0 || L.marker.ptr == L.out.ptr;
      // tagged hand-over (TAG, one tile per CTA): read the previous pass's
      // plane, write this pass's; no epochs
      const bool tagged = TAG && L.tagged != nullptr && ntiles <= (int)gridDim.x;
      const unsigned long long *tin = tagged && p > 0 ? L.tagged + (size_t)((p - 1) & 1) * L.tplane : nullptr;
      unsigned long long *tout = tagged && p + 1 < G.total_passes ? L.tagged + (size_t)(p & 1) * L.tplane : nullptr;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int ty = t / L.tiles_x, tx = t - ty * L.tiles_x;
        if (p > 0 && !tagged) {
          if (warp == 0 &&
              !wait_neighbours(L.epoch, ty, tx, L.tiles_y, L.tiles_x, L.fault ? p + (1 << 28) : p, lane,
                               L.wait_ns) &&
              lane == 0)
            record_status(L.status, GEO_ERR_TIMEOUT);
          __syncthreads();
        }
        const int64_t ty0 = (int64_t)ty * L.TH, tx0 = (int64_t)tx * L.TW;
        const bool ok =
            op == DILATE ? prog_tile<PD, TAG>(L, src, dst, src_cg, tin, tout, (unsigned)p, ty0, tx0, S,
                                              &xbuf[0][0][0][0], (NW + 2) * 2 * RWID, &xbar, parity, lane, warp, w, m)
                         : prog_tile<PE, TAG>(L, src, dst, src_cg, tin, tout, (unsigned)p, ty0, tx0, S,
                                              &xbuf[0][0][0][0], (NW + 2) * 2 * RWID, &xbar, parity, lane, warp, w, m);
        if (!ok) record_status(L.status, GEO_ERR_TIMEOUT);
        if (p + 1 < G.total_passes && !tagged) {
          __syncthreads();
          if (threadIdx.x == 0) st_release_u32(reinterpret_cast<unsigned *>(L.epoch) + t, (unsigned)(p + 1));
        }
      }
    }
  }
}

template <template <int> class RP, bool TAG = false>
int launch_prog(const TileLaunch &L, const Program &G, int grid, cudaStream_t s) {
  void *k = (void *)prog_kernel<RP, TAG>;
  const size_t smem = rr_smem_bytes<RP<DILATE>>();
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GEO_ERR_CUDA;
  TileLaunch a = L;
  Program g = G;
  void *args[] = {(void *)&a, (void *)&g};
  return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(RP<DILATE>::NW * 32), args, smem, s) == cudaSuccess
             ? GEO_OK
             : GEO_ERR_CUDA;
}

Plane prog_plane(const void *p, int64_t pitch_b, size_t va) {
  Plane q;
  q.ptr = (char *)p;
  q.pitch_b = pitch_b;
  q.vec_ok = (p != nullptr && ((uintptr_t)p % va) == 0 && pitch_b % (int64_t)va == 0) ? 1 : 0;
  q.bstride = 0;
  return q;
}

// Run the unmasked 8-connected runs (op[i], steps[i]) on f into out (which
// may equal f), at most kMaxRuns per launch.
int run_program(int dt, const void *f, void *out, int64_t H, int64_t W, int64_t pitch, const int *ops,
                const int64_t *steps, int nruns, cudaStream_t s) {
  int64_t total = 0;
  for (int i = 0; i < nruns; ++i) total += steps[i];
  Plan P;
  int rc = plan_rr(dt, DILATE, 4, 8, H, W, total, &P);
  if (rc != GEO_OK) return rc;
  int *status = nullptr;
  rc = device_status_word(&status);
  if (rc != GEO_OK) return rc;
  const int es = dt == GEO_U8 ? 1 : dt == GEO_F32 ? 4 : 8;
  const size_t va = (size_t)(dt == GEO_F64 ? 2 : 4) * es;  // the register kernel's CW pixels
  const int64_t spitch_b = ((W * es + 15) / 16) * 16;
  const size_t ntiles = (size_t)P.tiles_x * P.tiles_y;
  const size_t ctl_b = 256 + ((ntiles * sizeof(int) + 255) / 256) * 256;
  // uint8 programs with one tile per CTA hand the passes over in two planes
  // of tagged words (as the uint8 chains do; GEOMORPH_TAGGED=0: off), zeroed
  // before each launch together with the control words
  const char *tg = getenv("GEOMORPH_TAGGED");
  const bool tagged = dt == GEO_U8 && ntiles <= (size_t)P.grid && !single_tile(P, 1) && P.K % 4 == 0 &&
                      P.TW % 4 == 0 && !(tg && strcmp(tg, "0") == 0);
  const int64_t tpitch = (W + 3) / 4;
  const size_t tag_b = tagged ? ((2 * (size_t)tpitch * (size_t)H * 8 + 255) / 256) * 256 : 0;
  void *scratch = nullptr;
  rc = pool_alloc(&scratch, ctl_b + tag_b + (size_t)spitch_b * H, s);
  if (rc != GEO_OK) return rc;
  const void *src = f;
  for (int r0 = 0; r0 < nruns && rc == GEO_OK; r0 += kMaxRuns) {
    Program G;
    memset(&G, 0, sizeof(G));
    for (int i = r0; i < nruns && G.nruns < kMaxRuns; ++i) {
      G.op[G.nruns] = ops[i];
      G.steps[G.nruns] = steps[i];
      G.npasses[G.nruns] = (int)rr_passes(steps[i], single_tile(P, 1) ? 0 : P.K);
      G.total_passes += G.npasses[G.nruns];
      ++G.nruns;
    }
    if (G.total_passes == 0) {
      if (src != out &&
          cudaMemcpy2DAsync(out, pitch * es, src, pitch * es, W * es, H, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        rc = GEO_ERR_CUDA;
      src = out;
      continue;
    }
    // in place: the first pass must not write the buffer it reads, so the
    // pass count must be even (the last run takes one more, shorter pass)
    if (src == out && (G.total_passes & 1)) {
      ++G.npasses[G.nruns - 1];
      ++G.total_passes;
    }
    if (cudaMemsetAsync(scratch, 0, ctl_b + tag_b, s) != cudaSuccess) {
      rc = GEO_ERR_CUDA;
      break;
    }
    TileLaunch L;
    memset(&L, 0, sizeof(L));
    L.marker = prog_plane(src, pitch * es, va);
    L.mask = prog_plane(nullptr, 0, 1);
    L.out = prog_plane(out, pitch * es, va);
    L.scratch = prog_plane((char *)scratch + ctl_b + tag_b, spitch_b, va);
    L.H = H;
    L.W = W;
    L.TH = P.TH;
    L.TW = P.TW;
    L.K = P.K;
    L.tiles_x = P.tiles_x;
    L.tiles_y = P.tiles_y;
    L.mode = MODE_CHAIN;
    L.batch = 1;
    L.epoch = (int *)((char *)scratch + 256);
    L.ctl = (Control *)scratch;
    L.status = status;
    L.wait_ns = kWaitLimitNs;
    if (tagged && G.total_passes >= kTaggedMinPasses) {
      L.tagged = (unsigned long long *)((char *)scratch + ctl_b);
      L.tpitch = tpitch;
      L.tplane = tpitch * H;
    }
    rc = dt == GEO_U8 ? (L.tagged ? launch_prog<SU8, true>(L, G, P.grid, s) : launch_prog<SU8>(L, G, P.grid, s))
         : dt == GEO_F32 ? launch_prog<SF32>(L, G, P.grid, s)
                         : launch_prog<SF64>(L, G, P.grid, s);
    src = out;
  }
  if (pool_free(scratch, s) != GEO_OK && rc == GEO_OK) rc = GEO_ERR_CUDA;
  return rc;
}

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
  const int ops[2] = {first, first == ERODE ? DILATE : ERODE};
  const int64_t steps[2] = {s, s};
  return run_program(dt, f, out, H, W, pitch, ops, steps, 2, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// granulometry in one launch per size: gamma_k = delta_k(eps_k(f)) (Eq. 16)
// with eps_k = eps_1(eps_{k-1}) kept from size to size (Eq. 17's G_k needs
// only the sum of gamma_k, so gamma_k itself is never stored)
// ---------------------------------------------------------------------------

// One tile per CTA and pass, tiles independent within the launch: the region
// of eps_{k-1} with a halo of at least k + 1 (gran_halo), one erosion step (its interior is
// eps_k, stored for size k + 1), then k dilation steps on the same
// registers; the interior of the result is gamma_k, summed into partial[t].
// Between the two operations the rows beyond the region take the dilation's
// identity and the region's cells outside the image are clamped to it.
template <template <int> class RP>
__global__ void __launch_bounds__(RP<DILATE>::NW * 32, 1) gran_kernel(const TileLaunch L, int k,
                                                                       double *__restrict__ partial) {
  using PD = RP<DILATE>;
  using PE = RP<ERODE>;
  using RE = RR<PE>;
  using RD = RR<PD>;
  using Wd = typename PD::Wd;
  constexpr int CW = PD::CW, RW = PD::RW, NW = PD::NW, RWID = 32 * CW, PH = RW * PD::BANDS;
  extern __shared__ __align__(16) char rr_dyn[];
  Wd(*xbuf)[NW + 2][2][RWID] = reinterpret_cast<Wd(*)[NW + 2][2][RWID]>(rr_dyn);
  __shared__ __align__(8) uint64_t xbar;
  __shared__ double red[NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) mbar_init(&xbar, NW * 32);
  const int K = L.K, TH = L.TH, TW = L.TW;
  const int ntiles = L.tiles_x * L.tiles_y;
  int parity = 0;
  bool ok = true;
  Wd w[RW][CW], m[RW][CW];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int ty = t / L.tiles_x, tx = t - ty * L.tiles_x;
    const int64_t ty0 = (int64_t)ty * TH, tx0 = (int64_t)tx * TW;
    const int64_t gy0 = ty0 - K + warp * PH, gx = tx0 - K + lane * CW;
    __syncthreads();  // the previous tile's steps are done with the exchange rows
    for (int i = threadIdx.x; i < 2 * 2 * RWID; i += NW * 32) {
      const int par = i / (2 * RWID), rest = i % (2 * RWID);
      (&xbuf[par][0][0][0])[rest] = PE::identw();
      (&xbuf[par][NW + 1][0][0])[rest] = PE::identw();
    }
    __syncthreads();
    RE::load_words(L.marker, L.H, L.W, gy0, gx, true, false, w);
    RE::load_words(L.marker, L.H, L.W, gy0, gx, false, true, m);  // the erosion's virtual mask
    ok &= RE::template step<8>(w, m, &xbuf[parity][0][0][0], &xbar, parity, lane, warp);
    parity ^= 1;
    RE::store(w, L.out, L.out, false, L.H, L.W, ty0, tx0, K, TH, TW, lane, warp);  // eps_k
    __syncthreads();  // every warp past the erosion step's exchange
    for (int i = threadIdx.x; i < 2 * 2 * RWID; i += NW * 32) {
      const int par = i / (2 * RWID), rest = i % (2 * RWID);
      (&xbuf[par][0][0][0])[rest] = PD::identw();
      (&xbuf[par][NW + 1][0][0])[rest] = PD::identw();
    }
    __syncthreads();
    RD::load_words(L.marker, L.H, L.W, gy0, gx, false, true, m);  // the dilation's virtual mask
#pragma unroll
    for (int r = 0; r < RW; ++r)
#pragma unroll
      for (int c = 0; c < CW; ++c) w[r][c] = PD::clamp(w[r][c], m[r][c]);
    for (int j = 0; j < k; ++j) {
      ok &= RD::template step<8>(w, m, &xbuf[parity][0][0][0], &xbar, parity, lane, warp);
      parity ^= 1;
    }
    // sum of gamma_k over the tile's interior cells inside the image
    double acc = 0.0;
#pragma unroll
    for (int b = 0; b < PD::BANDS; ++b)
#pragma unroll
      for (int r = 0; r < RW; ++r) {
        const int Y = warp * PH + b * RW + r;
        if (Y < K || Y >= K + TH || ty0 + (Y - K) >= L.H) continue;
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          const int X = lane * CW + c;
          if (X < K || X >= K + TW || tx0 + (X - K) >= L.W) continue;
          acc += (double)PD::from_px(PD::get(w[r][c], b));
        }
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int i = 0; i < NW; ++i) sum += red[i];
      partial[t] = sum;
    }
  }
  if (!ok && threadIdx.x == 0) record_status(L.status, GEO_ERR_TIMEOUT);
}

// G[1 + b] = sum of partial[b * stride .. b * stride + stride) in a fixed tree
// order (one block per size; unused entries are zero)
__global__ void __launch_bounds__(kSumBlocks) gran_final(const double *__restrict__ partial, int stride, double *G) {
  __shared__ double red[kSumBlocks];
  const double *p = partial + (size_t)blockIdx.x * stride;
  double acc = 0.0;
  for (int i = threadIdx.x; i < stride; i += kSumBlocks) acc += p[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kSumBlocks / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) G[1 + blockIdx.x] = red[0];
}

// The largest size the fused launch takes for an element type: the halo
// within a third of the register region's shorter side (as the planner's
// K), so that the interior keeps at least a third of it; and the per-tile
// sums' stride (the tiles of the largest size, which has the most).
// The halo is k + 1 rounded up to whole lanes (CW columns), as every pass
// of the register kernel: a lane's columns then lie wholly in the interior
// or wholly in the halo.
template <template <int> class RP>
int gran_halo(int64_t k) {
  constexpr int CW = RP<DILATE>::CW;
  return (int)((k + 1 + CW - 1) / CW * CW);
}
template <template <int> class RP>
int gran_fused_max() {
  using PD = RP<DILATE>;
  constexpr int RWID = 32 * PD::CW, RHGT = PD::NW * PD::RW * PD::BANDS;
  return (RWID < RHGT ? RWID : RHGT) / 3 / PD::CW * PD::CW - 1;
}
template <template <int> class RP>
int gran_fused_tiles(int64_t H, int64_t W, int64_t smax) {
  using PD = RP<DILATE>;
  constexpr int RWID = 32 * PD::CW, RHGT = PD::NW * PD::RW * PD::BANDS;
  const int K = gran_halo<RP>(smax);
  return (int)(((H + (RHGT - 2 * K) - 1) / (RHGT - 2 * K)) * ((W + (RWID - 2 * K) - 1) / (RWID - 2 * K)));
}

template <template <int> class RP>
int gran_fused(const void *f, int64_t H, int64_t W, int64_t pitch, int64_t smax, double *G, cudaStream_t s,
               char *eps_a, char *eps_b, double *partial, int stride, int *status) {
  using PD = RP<DILATE>;
  constexpr int RWID = 32 * PD::CW, RHGT = PD::NW * PD::RW * PD::BANDS;
  void *kern = (void *)gran_kernel<RP>;
  const size_t smem = rr_smem_bytes<PD>();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GEO_ERR_CUDA;
  const int es = (int)sizeof(typename PD::G);
  const size_t va = (size_t)PD::CW * es;
  const void *src = f;
  for (int64_t k = 1; k <= smax; ++k) {
    char *dst = (k & 1) ? eps_a : eps_b;
    TileLaunch L;
    memset(&L, 0, sizeof(L));
    L.K = gran_halo<RP>(k);
    L.TH = RHGT - 2 * L.K;
    L.TW = RWID - 2 * L.K;
    L.tiles_x = (int)((W + L.TW - 1) / L.TW);
    L.tiles_y = (int)((H + L.TH - 1) / L.TH);
    L.marker = prog_plane(src, pitch * es, va);
    L.out = prog_plane(dst, pitch * es, va);
    L.mask = prog_plane(nullptr, 0, 1);
    L.H = H;
    L.W = W;
    L.status = status;
    L.wait_ns = kWaitLimitNs;
    const int ntiles = L.tiles_x * L.tiles_y;
    if (ntiles > stride) return GEO_ERR_ARG;
    TileLaunch a = L;
    int kk = (int)k;
    double *pk = partial + (size_t)(k - 1) * stride;
    void *args[] = {(void *)&a, (void *)&kk, (void *)&pk};
    if (cudaLaunchKernel(kern, dim3(ntiles), dim3(PD::NW * 32), args, smem, s) != cudaSuccess) return GEO_ERR_CUDA;
    src = dst;
  }
  gran_final<<<(unsigned)smax, kSumBlocks, 0, s>>>(partial, stride, G);
  return cudaGetLastError() == cudaSuccess ? GEO_OK : GEO_ERR_CUDA;
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
  // which leaves E 1, D 2, E 3, D 4, ..., D 2s, E s, all in one program
  std::vector<int> ops;
  std::vector<int64_t> steps;
  int cur_op = ERODE;
  int64_t run = 0;
  for (int64_t k = 1; k <= s; ++k) {
    const int seq[4] = {ERODE, DILATE, DILATE, ERODE};
    for (int i = 0; i < 4; ++i) {
      if (seq[i] == cur_op) {
        run += k;
      } else {
        ops.push_back(cur_op);
        steps.push_back(run);
        cur_op = seq[i];
        run = k;
      }
    }
  }
  ops.push_back(cur_op);
  steps.push_back(run);
  return run_program(dtype, f, out, H, W, pitch, ops.data(), steps.data(), (int)ops.size(), (cudaStream_t)stream);
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
  // scratch: [partial sums][eps_s(f)][gamma_s(f) or eps_s(f)], images with
  // f's pitch; the fused form's per-tile sums of every size after them
  const size_t part_b = kSumBlocks * sizeof(double);
  const size_t img_b = (((size_t)((H - 1) * pitch + W) * es) + 255) / 256 * 256;
  // Sizes up to gran_fused_max run one launch each (erosion step, dilation
  // steps and the interior sums of every tile together); larger ones go
  // through the window calls, one erosion step, one window and one sum each.
  const int fmax = dtype == GEO_U8 ? gran_fused_max<SU8>() : dtype == GEO_F32 ? gran_fused_max<SF32>()
                                                                              : gran_fused_max<SF64>();
  const bool fused = smax >= 1 && smax <= fmax;
  const int stride = !fused ? 0
                     : dtype == GEO_U8  ? gran_fused_tiles<SU8>(H, W, smax)
                     : dtype == GEO_F32 ? gran_fused_tiles<SF32>(H, W, smax)
                                        : gran_fused_tiles<SF64>(H, W, smax);
  void *scratch = nullptr;
  int rc = pool_alloc(&scratch, part_b + 2 * img_b + (size_t)smax * stride * sizeof(double), s);
  if (rc != GEO_OK) return rc;
  double *partial = (double *)scratch;
  char *ero = (char *)scratch + part_b, *gam = ero + img_b;
  double *tile_sums = (double *)(gam + img_b);
  rc = image_sum(dtype, f, H, W, pitch, partial, G, s);
  if (fused && rc == GEO_OK) {
    int *status = nullptr;
    rc = device_status_word(&status);
    if (rc == GEO_OK && cudaMemsetAsync(tile_sums, 0, (size_t)smax * stride * sizeof(double), s) != cudaSuccess)
      rc = GEO_ERR_CUDA;
    if (rc == GEO_OK)
      rc = dtype == GEO_U8 ? gran_fused<SU8>(f, H, W, pitch, smax, G, s, ero, gam, tile_sums, stride, status)
           : dtype == GEO_F32 ? gran_fused<SF32>(f, H, W, pitch, smax, G, s, ero, gam, tile_sums, stride, status)
                              : gran_fused<SF64>(f, H, W, pitch, smax, G, s, ero, gam, tile_sums, stride, status);
  }
  for (int64_t k = 1; !fused && k <= smax && rc == GEO_OK; ++k) {
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
