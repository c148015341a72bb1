// Quasi-distance transform (Section 2, Eq. 13-15; Section 3.8, Algorithm 6)
// on the register-resident 3x3 engine of geo_rr.cuh.
//
// Part 1, d(f) of Eq. 13 as Algorithm 6 builds it: the chain of unmasked
// erosions eps_1 and, for every pixel, the largest residual
// eps_{j-1}(f) - eps_j(f) so far together with the first erosion j that
// attains it. The pair lives in one 32-bit key per pixel,
//     key = r << 16 | (65535 - d),
// and taking the maximum of the key and each erosion's candidate is exactly
// Algorithm 6's strictly-larger update: a larger residual wins, an equal one
// keeps the earlier j (whose 65535 - j is larger). The initial state r = 0,
// d = 0 is the key 0x0000ffff, which no zero residual exceeds. Keys are
// decoded into the caller's r (uint8) and d (int32) images and re-encoded
// when a tile is reloaded.
//
// Part 2, Eq. 14-15: eta applied to d until a step changes nothing. For
// integer images eta(g) (eps_1(g) + 1 where g - eps_1(g) > 1, g elsewhere) is
// min(g, eps_1(g) + 1); it runs as a reconstruction of the register kernel
// whose per-word rule is that minimum in place of the mask clamp (RD32).
#include <cstring>

#include "geo_rr.cuh"

namespace geo {

// ---------------------------------------------------------------------------
// distances of the eta iteration: int32 in memory (0 .. 0x7ffe), held like
// the uint8 pixels as two u16 lanes of one word (rows r and r + RW)
// ---------------------------------------------------------------------------
struct RD32 {
  using Wd = uint32_t;
  using Px = uint32_t;
  using G = int32_t;
  static constexpr int BANDS = 2, CW = 4, RW = GEO_RR_U8_RW, NW = GEO_RR_U8_NW, GS = 4;
  static constexpr uint32_t kIdent = 0x7fffu;  // above every distance, and +1 stays inside the lane
  static constexpr bool PAIRS = true;
  static constexpr int FMA = 0;
  __device__ static Wd e2(Wd a, Wd b) { return umin2(a, b); }
  __device__ static Wd e2h(Wd a, Wd b) { return umin2(a, b); }
  __device__ static Wd e2m(Wd a, Wd b) { return umin2(a, b); }
  __device__ static Wd ext3(Wd a, Wd b, Wd c) { return umin2(umin2(a, b), c); }
  __device__ static Wd ext3h(Wd a, Wd b, Wd c) { return ext3(a, b, c); }
  __device__ static Wd clamp(Wd v, Wd m) { return umax2(v, m); }
  // eta on both lanes: min(old, eps_1 + 1), then the virtual mask keeps the
  // cells outside the image at the identity
  __device__ static Wd apply(Wd v, Wd m, Wd old) { return umax2(umin2(old, v + 0x00010001u), m); }
  __device__ static Px ident() { return kIdent; }
  __device__ static Px anti() { return 0u; }
  __device__ static Wd identw() { return kIdent * 0x00010001u; }
  __device__ static Wd make(Px lo, Px hi) { return lo | (hi << 16); }
  __device__ static Px get(Wd w, int band) { return band ? (w >> 16) : (w & 0xffffu); }
  __device__ static Wd up(Wd above, Wd own_last) { return __funnelshift_l(above, own_last, 16); }
  __device__ static Wd down(Wd own_first, Wd below) { return __funnelshift_r(own_first, below, 16); }
  __device__ static Px to_px(G g) { return (Px)g; }
  __device__ static G from_px(Px p) { return (G)p; }
  __device__ static uint4 pack(const Wd (&v)[CW]) { return make_uint4(v[0], v[1], v[2], v[3]); }
  __device__ static void unpack(uint4 u, Wd (&v)[CW]) {
    v[0] = u.x;
    v[1] = u.y;
    v[2] = u.z;
    v[3] = u.w;
  }
  using Raw = int4;
  __device__ static Raw load_raw(const char *p, bool cg) {
    return cg ? __ldcg(reinterpret_cast<const int4 *>(p)) : __ldg(reinterpret_cast<const int4 *>(p));
  }
  __device__ static void unpack_raw(Raw x, Px (&v)[CW]) {
    v[0] = (Px)x.x;
    v[1] = (Px)x.y;
    v[2] = (Px)x.z;
    v[3] = (Px)x.w;
  }
  __device__ static void load_vec(const char *p, bool cg, Px (&v)[CW]) { unpack_raw(load_raw(p, cg), v); }
  __device__ static void store_vec(char *p, const Px (&v)[CW]) {
    __stcg(reinterpret_cast<int4 *>(p), make_int4((int)v[0], (int)v[1], (int)v[2], (int)v[3]));
  }
  __device__ static bool differs_vec(const char *p, const Px (&v)[CW]) {
    const int4 o = __ldcg(reinterpret_cast<const int4 *>(p));
    return (o.x != (int)v[0]) | (o.y != (int)v[1]) | (o.z != (int)v[2]) | (o.w != (int)v[3]);
  }
};

namespace {

// the image of part 1: uint8, erosion, no mask; the clamp runs on the FMA
// pipe because the observer's key updates load the ALU pipe
using QP = RU8<ERODE, GEO_RR_U8_RW, GEO_RR_U8_NW, 1>;

// Residual/erosion keys of one lane's pixels: k[band][word row][column]. As
// the step observer it folds each written word's two residuals into the
// keys; cs = 65535 - j for the erosion j being applied.
struct QdtKeys {
  static constexpr int RW = QP::RW, CW = QP::CW;
  uint32_t k[2][RW][CW];
  uint32_t cs;
  __device__ __forceinline__ void operator()(int r, int c, uint32_t old, uint32_t nw) {
    const uint32_t res = old - nw;  // both u16 lanes: nw <= old (the erosion includes the centre), no borrow
    k[0][r][c] = max(k[0][r][c], __byte_perm(res, cs, 0x1054));  // (res_lo << 16) | cs
    k[1][r][c] = max(k[1][r][c], __byte_perm(res, cs, 0x3254));  // (res_hi << 16) | cs
  }
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int r = 0; r < RW; ++r)
#pragma unroll
        for (int c = 0; c < CW; ++c) k[b][r][c] = 0x0000ffffu;
  }
};

// Visit the interior pixels of a lane (the ones a pass stores): fn(b, r, c,
// row pointer offset gy, column gx + c), skipping columns past the image.
template <class Fn>
__device__ __forceinline__ void for_interior(const TileLaunch &L, int64_t ty0, int64_t tx0, int lane, int warp,
                                             Fn fn) {
  constexpr int CW = QP::CW, RW = QP::RW, PH = 2 * RW;
  const int K = L.K, X = lane * CW;
  if (X < K || X + CW > K + L.TW) return;
  const int64_t gx = tx0 + (X - K);
  if (gx >= L.W) return;
#pragma unroll
  for (int b = 0; b < 2; ++b) {
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      const int Y = warp * PH + b * RW + r;
      if (Y < K || Y >= K + L.TH) continue;
      const int64_t gy = ty0 + (Y - K);
      if (gy >= L.H) continue;
      fn(b, r, gy, gx);
    }
  }
}

__device__ __forceinline__ void keys_store(const QdtKeys &q, const TileLaunch &L, const Plane &Rp, const Plane &Dp,
                                           int64_t ty0, int64_t tx0, int lane, int warp) {
  constexpr int CW = QP::CW;
  for_interior(L, ty0, tx0, lane, warp, [&](int b, int r, int64_t gy, int64_t gx) {
    uint8_t *rp = reinterpret_cast<uint8_t *>(Rp.ptr + gy * Rp.pitch_b) + gx;
    int32_t *dp = reinterpret_cast<int32_t *>(Dp.ptr + gy * Dp.pitch_b) + gx;
    uint32_t rv[CW];
    int32_t dv[CW];
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      rv[c] = q.k[b][r][c] >> 16;
      dv[c] = 65535 - (int32_t)(q.k[b][r][c] & 0xffffu);
    }
    if (gx + CW <= L.W && Rp.vec_ok && Dp.vec_ok) {
      __stcg(reinterpret_cast<unsigned *>(rp), rv[0] | (rv[1] << 8) | (rv[2] << 16) | (rv[3] << 24));
      __stcg(reinterpret_cast<int4 *>(dp), make_int4(dv[0], dv[1], dv[2], dv[3]));
    } else {
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        if (gx + c < L.W) {
          __stcg(rp + c, (uint8_t)rv[c]);
          __stcg(dp + c, dv[c]);
        }
      }
    }
  });
}

__device__ __forceinline__ void keys_load(QdtKeys &q, const TileLaunch &L, const Plane &Rp, const Plane &Dp,
                                          int64_t ty0, int64_t tx0, int lane, int warp) {
  constexpr int CW = QP::CW;
  q.init();
  for_interior(L, ty0, tx0, lane, warp, [&](int b, int r, int64_t gy, int64_t gx) {
    const uint8_t *rp = reinterpret_cast<const uint8_t *>(Rp.ptr + gy * Rp.pitch_b) + gx;
    const int32_t *dp = reinterpret_cast<const int32_t *>(Dp.ptr + gy * Dp.pitch_b) + gx;
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      if (gx + c < L.W) {
        const uint32_t rv = __ldcg(rp + c);
        const int32_t dv = __ldcg(dp + c);
        q.k[b][r][c] = (rv << 16) | (uint32_t)(65535 - dv);
      }
    }
  });
}

// Part 1. Chain of L.steps unmasked erosions of L.marker, passes of K steps
// synchronised point to point by the per-tile epochs as in rr_kernel; the
// image ping-pongs between L.out and L.scratch (both library scratch), the
// keys go to Rp / Dp. With one tile per CTA and L.tagged set, the passes
// hand the image over in tagged words instead (as the uint8 chains of
// rr_kernel do: no epochs, release fence or second round trip; the same
// write-after-read argument holds, every tile's stores depending on its
// tag-checked loads).
template <int CONN>
__global__ void __launch_bounds__(QP::NW * 32, 1) qdt_kernel(const TileLaunch L, const Plane Rp, const Plane Dp) {
  using R = RR<QP>;
  using Wd = typename QP::Wd;
  constexpr int CW = R::CW, RW = R::RW, NW = R::NW, PH = R::PH, RWID = R::RWID;
  extern __shared__ __align__(16) char rr_dyn[];
  Wd(*xbuf)[NW + 2][2][RWID] = reinterpret_cast<Wd(*)[NW + 2][2][RWID]>(rr_dyn);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int K = L.K, TH = L.TH, TW = L.TW;
  const int ntiles = L.tiles_x * L.tiles_y;
  const bool resident = ntiles <= (int)gridDim.x;  // one tile per CTA: keys stay in registers
  const bool tagged = resident && L.tagged != nullptr;

  __shared__ __align__(8) uint64_t xbar;
  if (threadIdx.x == 0) mbar_init(&xbar, NW * 32);
  for (int i = threadIdx.x; i < 2 * 2 * RWID; i += NW * 32) {
    const int par = i / (2 * RWID), rest = i % (2 * RWID);
    (&xbuf[par][0][0][0])[rest] = QP::identw();
    (&xbuf[par][NW + 1][0][0])[rest] = QP::identw();
  }
  __syncthreads();

  Wd w[RW][CW], m[RW][CW];
  QdtKeys q;
  int parity = 0;
  const int64_t base = L.steps / L.npasses, extra = L.steps % L.npasses;
  for (int pass = 0; pass < L.npasses; ++pass) {
    const int S = (int)(base + (pass < extra ? 1 : 0));
    const int64_t j0 = pass * base + (pass < extra ? pass : extra);  // erosions before this pass
    const Plane srcP = pass == 0 ? L.marker : (((pass - 1) & 1) ? L.scratch : L.out);
    const Plane dstP = (pass & 1) ? L.scratch : L.out;
    const bool last = pass + 1 == L.npasses;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int ty = t / L.tiles_x, tx = t - ty * L.tiles_x;
      const int64_t ty0 = (int64_t)ty * TH, tx0 = (int64_t)tx * TW;
      const int64_t gy0 = ty0 - K + warp * PH, gx = tx0 - K + lane * CW;
      if (pass > 0 && !tagged) {
        if (warp == 0 && !wait_neighbours(L.epoch, ty, tx, L.tiles_y, L.tiles_x, pass, lane, L.wait_ns) && lane == 0)
          record_status(L.status, GEO_ERR_TIMEOUT);
        __syncthreads();
      }
      if (tagged && pass > 0) {
        if (!R::load_tagged(R::tplane(L, (pass - 1) & 1), L.tpitch, L.H, L.W, gy0, gx, (unsigned)pass, L.wait_ns, w))
          record_status(L.status, GEO_ERR_TIMEOUT);
      } else {
        R::load_words(srcP, L.H, L.W, gy0, gx, pass > 0, false, w);
      }
      if (pass == 0 || !resident) R::load_words(L.mask, L.H, L.W, gy0, gx, false, true, m);
      if (pass == 0) q.init();
      else if (!resident) keys_load(q, L, Rp, Dp, ty0, tx0, lane, warp);
      bool ok = true;
      for (int j = 0; j < S; ++j) {
        q.cs = 65535u - (uint32_t)(j0 + j + 1);
        ok &= R::template step<CONN>(w, m, &xbuf[parity][0][0][0], &xbar, parity, lane, warp, q);
        parity ^= 1;
      }
      if (!ok) record_status(L.status, GEO_ERR_TIMEOUT);
      if (last || !resident) keys_store(q, L, Rp, Dp, ty0, tx0, lane, warp);
      if (!last && tagged) {
        R::store_tagged(w, R::tplane(L, pass & 1), L.tpitch, L.H, L.W, ty0, tx0, K, TH, TW, (unsigned)(pass + 1), lane,
                        warp);
      } else if (!last) {
        R::store(w, dstP, dstP, false, L.H, L.W, ty0, tx0, K, TH, TW, lane, warp);
        __syncthreads();
        if (threadIdx.x == 0) st_release_u32(reinterpret_cast<unsigned *>(L.epoch) + t, (unsigned)(pass + 1));
      }
    }
  }
}

template <int CONN>
void *qdt_kernel_ptr() {
  return (void *)qdt_kernel<CONN>;
}

}  // namespace

// host side of the eta reconstruction (run_chain with the internal dtype GEO_D32)
int launch_rr_d32(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid) {
  if (op != ERODE) return GEO_ERR_ARG;
  void *k = conn == 8 ? (void *)rr_kernel<RD32, 8> : (void *)rr_kernel<RD32, 4>;
  const size_t smem = rr_smem_bytes<RD32>();
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GEO_ERR_CUDA;
  TileLaunch arg = L;
  void *args[] = {(void *)&arg};
  return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(RD32::NW * 32), args, smem, s) == cudaSuccess ? GEO_OK
                                                                                                      : GEO_ERR_CUDA;
}

int occupancy_rr_d32(int op, int conn, int *bps) {
  (void)op;
  void *k = conn == 8 ? (void *)rr_kernel<RD32, 8> : (void *)rr_kernel<RD32, 4>;
  const size_t smem = rr_smem_bytes<RD32>();
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GEO_ERR_CUDA;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, RD32::NW * 32, smem) == cudaSuccess ? GEO_OK
                                                                                                   : GEO_ERR_CUDA;
}

}  // namespace geo

using namespace geo;

namespace {

int64_t qdt_chain_steps(int64_t H, int64_t W, int conn) {
  if (H == 0 || W == 0) return 0;
  return conn == 8 ? (H > W ? H : W) - 1 : H + W - 2;
}

bool spans_overlap(const void *a, size_t na, const void *b, size_t nb) {
  const char *x = (const char *)a, *y = (const char *)b;
  return x < y + nb && y < x + na;
}

}  // namespace

extern "C" {

int geo_qdt(geo_dtype dtype, const void *f, void *r, int32_t *d, int32_t *d_l1, int64_t height, int64_t width,
            int64_t pitch, int conn, void *stream) {
  if (dtype != GEO_U8) return GEO_ERR_DTYPE;
  const int64_t H = height, W = width;
  if (H < 0 || W < 0 || pitch < W || (conn != 4 && conn != 8)) return GEO_ERR_ARG;
  if (H == 0 || W == 0) return GEO_OK;
  if (!f || !r || !d) return GEO_ERR_ARG;
  if (((uintptr_t)d % 4) || (d_l1 && ((uintptr_t)d_l1 % 4))) return GEO_ERR_ALIGN;
  const int64_t S = qdt_chain_steps(H, W, conn);
  if (S > 32766) return GEO_ERR_ARG;  // distances must stay below the u16 lane's identity
  const size_t n8 = (size_t)((H - 1) * pitch + W), n32 = n8 * 4;
  if (spans_overlap(f, n8, r, n8) || spans_overlap(f, n8, d, n32) || spans_overlap(r, n8, d, n32)) return GEO_ERR_ARG;
  if (d_l1 && d_l1 != d && (spans_overlap(d_l1, n32, f, n8) || spans_overlap(d_l1, n32, r, n8) ||
                            spans_overlap(d_l1, n32, d, n32)))
    return GEO_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;

  if (S == 0) {  // a single pixel: no erosion lowers it
    if (cudaMemsetAsync(r, 0, 1, s) != cudaSuccess || cudaMemsetAsync(d, 0, 4, s) != cudaSuccess) return GEO_ERR_CUDA;
    if (d_l1 && cudaMemsetAsync(d_l1, 0, 4, s) != cudaSuccess) return GEO_ERR_CUDA;
    return GEO_OK;
  }

  int *status = nullptr;
  int rc = device_status_word(&status);
  if (rc != GEO_OK) return rc;
  Plan P;
  rc = plan_rr(GEO_U8, ERODE, 5, conn, H, W, S, &P);
  if (rc != GEO_OK) return rc;

  // scratch: [control 256 B][per-tile epochs][two tagged planes][two image buffers]
  const int64_t spitch = ((W + 15) / 16) * 16;
  const size_t ntiles = (size_t)P.tiles_x * (size_t)P.tiles_y;
  const size_t ctl_b = 256 + ((ntiles * sizeof(int) + 255) / 256) * 256;
  const size_t img_b = ((size_t)spitch * (size_t)H + 255) / 256 * 256;
  const int64_t npasses = rr_passes(S, single_tile(P, 1) ? 0 : P.K);
  // one tile per CTA and several passes: the passes hand over in two zeroed
  // planes of tagged words (GEOMORPH_TAGGED=0: plain buffers and epochs)
  const char *tg = getenv("GEOMORPH_TAGGED");
  const bool tagged = ntiles <= (size_t)P.grid && npasses >= kTaggedMinPasses && P.K % 4 == 0 && P.TW % 4 == 0 &&
                      !(tg && strcmp(tg, "0") == 0);
  const int64_t tpitch = (W + 3) / 4;
  const size_t tag_b = tagged ? ((2 * (size_t)tpitch * (size_t)H * 8 + 255) / 256) * 256 : 0;
  void *scratch = nullptr;
  rc = pool_alloc(&scratch, ctl_b + tag_b + 2 * img_b, s);
  if (rc != GEO_OK) return rc;
  if (cudaMemsetAsync(scratch, 0, ctl_b + tag_b, s) != cudaSuccess) rc = GEO_ERR_CUDA;

  auto plane = [](const void *p, int64_t pitch_b, size_t va) {
    Plane q;
    q.ptr = (char *)p;
    q.pitch_b = pitch_b;
    q.vec_ok = (p != nullptr && ((uintptr_t)p % va) == 0 && pitch_b % (int64_t)va == 0) ? 1 : 0;
    q.bstride = 0;
    return q;
  };
  TileLaunch L;
  memset(&L, 0, sizeof(L));
  L.marker = plane(f, pitch, QP::CW);
  L.mask = plane(nullptr, 0, 1);
  L.out = plane((char *)scratch + ctl_b + tag_b, spitch, QP::CW);
  L.scratch = plane((char *)scratch + ctl_b + tag_b + img_b, spitch, QP::CW);
  L.H = H;
  L.W = W;
  L.TH = P.TH;
  L.TW = P.TW;
  L.K = P.K;
  L.tiles_x = P.tiles_x;
  L.tiles_y = P.tiles_y;
  L.mode = MODE_CHAIN;
  L.steps = S;
  L.npasses = (int)npasses;
  if (tagged) {
    L.tagged = (unsigned long long *)((char *)scratch + ctl_b);
    L.tpitch = tpitch;
    L.tplane = tpitch * H;
  }
  L.ctl = (Control *)scratch;
  L.epoch = (int *)((char *)scratch + 256);
  L.status = status;
  L.batch = 1;
  L.wait_ns = kWaitLimitNs;
  const Plane Rp = plane(r, pitch, QP::CW), Dp = plane(d, pitch * 4, QP::CW * 4);
  if (rc == GEO_OK) {
    void *k = conn == 8 ? qdt_kernel_ptr<8>() : qdt_kernel_ptr<4>();
    const size_t smem = rr_smem_bytes<QP>();
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      rc = GEO_ERR_CUDA;
    } else {
      void *args[] = {(void *)&L, (void *)&Rp, (void *)&Dp};
      if (cudaLaunchCooperativeKernel(k, dim3(P.grid), dim3(QP::NW * 32), args, smem, s) != cudaSuccess)
        rc = GEO_ERR_CUDA;
    }
  }
  if (pool_free(scratch, s) != GEO_OK && rc == GEO_OK) rc = GEO_ERR_CUDA;
  if (rc != GEO_OK || !d_l1) return rc;
  // part 2: the eta limit of d (Eq. 15), a reconstruction with the distance policy
  return run_chain_any(GEO_D32, d, nullptr, d_l1, H, W, pitch, conn, ERODE, MODE_REC, H * W + 1 + 1024, nullptr,
                       stream, 1);
}

}  // extern "C"
