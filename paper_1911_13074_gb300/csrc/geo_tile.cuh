// Persistent, temporally blocked tile kernel for geodesic 3x3 chains.
//
// One launch runs a whole chain (Eq. 4) or a whole reconstruction (Eq. 5).
// The image is cut into TH x TW tiles. A pass loads each tile plus a K-pixel
// halo of the current image into shared memory, applies S <= K elementary
// steps there (Eq. 3: separable 3-extreme along the row, then along the
// column (the decomposition of Section 3.1), then the clamp with the mask),
// and writes the tile interior back. The region that is still exact shrinks
// by one pixel per step, so after S steps the interior is exact. Passes are
// separated by a grid-wide barrier; reconstruction ORs a per-pass "changed"
// flag and stops after the first pass that changed nothing (Section 3.7,
// Algorithm 5 detects convergence the same way, per filter).
//
// Pixels outside the image hold the identity of the extreme in both the
// marker (lowest value for dilation) and the mask, so they never change and
// never win, which is the clipping w_1(p) of Section 2.
//
// Element policies keep pixels in shared memory in a form the sm_103a integer
// and FP32 pipes handle at full rate:
//   u8  -> u16 lanes, two pixels per 32-bit word, max.u16x2 / min.u16x2
//   f32 -> f32, three-input max.f32 / min.f32 for the 3-extremes
//   f64 -> order-preserving int64 keys (max.s64), exact for every double
//          except NaN and -0.0, which are outside the contract.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "geo_common.cuh"

namespace geo {

// ---------------------------------------------------------------------------
// element policies
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t umax2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t umin2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// u8 images: shared memory holds u16 lanes; a 16-byte chunk = 8 pixels.
template <int OP>
struct EU8 {
  using G = uint8_t;
  static constexpr int CE = 8;        // pixels per 16-byte chunk in shared memory
  static constexpr int GS = 1;        // bytes per pixel in global memory
  static constexpr int SS = 2;        // bytes per pixel in shared memory
  __device__ static uint32_t ext(uint32_t a, uint32_t b) { return OP == DILATE ? umax2(a, b) : umin2(a, b); }
  __device__ static uint32_t opp(uint32_t a, uint32_t b) { return OP == DILATE ? umin2(a, b) : umax2(a, b); }
  // identity of the extreme (never wins) and its opposite, as one u16 pixel
  __device__ static uint16_t ident() { return OP == DILATE ? 0 : 255; }
  __device__ static uint16_t anti() { return OP == DILATE ? 255 : 0; }
  __device__ static uint16_t to_s(uint8_t v) { return v; }
  __device__ static uint8_t from_s(uint16_t v) { return (uint8_t)v; }

  // horizontal 3-extreme of the chunk c given the 32-bit words just left
  // (its high lane is the left neighbour) and right (low lane) of it
  __device__ static uint4 hext(uint4 c, uint32_t left, uint32_t right) {
    uint4 h;
    h.x = ext(ext(__funnelshift_l(left, c.x, 16), c.x), __funnelshift_r(c.x, c.y, 16));
    h.y = ext(ext(__funnelshift_l(c.x, c.y, 16), c.y), __funnelshift_r(c.y, c.z, 16));
    h.z = ext(ext(__funnelshift_l(c.y, c.z, 16), c.z), __funnelshift_r(c.z, c.w, 16));
    h.w = ext(ext(__funnelshift_l(c.z, c.w, 16), c.w), __funnelshift_r(c.w, right, 16));
    return h;
  }
  __device__ static uint4 ext3(uint4 a, uint4 b, uint4 c) {
    return make_uint4(ext(ext(a.x, b.x), c.x), ext(ext(a.y, b.y), c.y), ext(ext(a.z, b.z), c.z),
                      ext(ext(a.w, b.w), c.w));
  }
  __device__ static uint4 clamp(uint4 v, uint4 m) {
    return make_uint4(opp(v.x, m.x), opp(v.y, m.y), opp(v.z, m.z), opp(v.w, m.w));
  }
  // words holding the neighbours of a chunk starting at shared address p
  __device__ static uint32_t left_word(const char *p) { return *(const uint32_t *)(p - 4); }
  __device__ static uint32_t right_word(const char *p) { return *(const uint32_t *)(p + 16); }
};

// f32 images: a chunk = 4 floats.
template <int OP>
struct EF32 {
  using G = float;
  static constexpr int CE = 4;
  static constexpr int GS = 4;
  static constexpr int SS = 4;
  __device__ static float e3(float a, float b, float c) { return OP == DILATE ? fmax3(a, b, c) : fmin3(a, b, c); }
  __device__ static float opp(float a, float b) { return OP == DILATE ? fminf(a, b) : fmaxf(a, b); }
  __device__ static float ident() { return OP == DILATE ? -__int_as_float(0x7f800000) : __int_as_float(0x7f800000); }
  __device__ static float anti() { return OP == DILATE ? __int_as_float(0x7f800000) : -__int_as_float(0x7f800000); }
  __device__ static float to_s(float v) { return v; }
  __device__ static float from_s(float v) { return v; }
  __device__ static uint4 hext(uint4 c, uint32_t left, uint32_t right) {
    float4 f = *reinterpret_cast<float4 *>(&c);
    float4 h;
    h.x = e3(__uint_as_float(left), f.x, f.y);
    h.y = e3(f.x, f.y, f.z);
    h.z = e3(f.y, f.z, f.w);
    h.w = e3(f.z, f.w, __uint_as_float(right));
    return *reinterpret_cast<uint4 *>(&h);
  }
  __device__ static uint4 ext3(uint4 a, uint4 b, uint4 c) {
    float4 x = *reinterpret_cast<float4 *>(&a), y = *reinterpret_cast<float4 *>(&b),
           z = *reinterpret_cast<float4 *>(&c), r;
    r.x = e3(x.x, y.x, z.x);
    r.y = e3(x.y, y.y, z.y);
    r.z = e3(x.z, y.z, z.z);
    r.w = e3(x.w, y.w, z.w);
    return *reinterpret_cast<uint4 *>(&r);
  }
  __device__ static uint4 clamp(uint4 v, uint4 m) {
    float4 x = *reinterpret_cast<float4 *>(&v), y = *reinterpret_cast<float4 *>(&m), r;
    r.x = opp(x.x, y.x);
    r.y = opp(x.y, y.y);
    r.z = opp(x.z, y.z);
    r.w = opp(x.w, y.w);
    return *reinterpret_cast<uint4 *>(&r);
  }
  __device__ static uint32_t left_word(const char *p) { return *(const uint32_t *)(p - 4); }
  __device__ static uint32_t right_word(const char *p) { return *(const uint32_t *)(p + 16); }
};

// f64 images: a chunk = 2 order-preserving int64 keys.
__device__ __forceinline__ long long f64_key(double d) {
  long long b = __double_as_longlong(d);
  return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double key_f64(long long k) {
  return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffLL));
}

template <int OP>
struct EF64 {
  using G = double;
  static constexpr int CE = 2;
  static constexpr int GS = 8;
  static constexpr int SS = 8;
  __device__ static long long e(long long a, long long b) { return OP == DILATE ? max(a, b) : min(a, b); }
  __device__ static long long opp(long long a, long long b) { return OP == DILATE ? min(a, b) : max(a, b); }
  __device__ static long long ident() { return OP == DILATE ? (long long)0x8000000000000000ULL : 0x7fffffffffffffffLL; }
  __device__ static long long anti() { return OP == DILATE ? 0x7fffffffffffffffLL : (long long)0x8000000000000000ULL; }
  __device__ static long long to_s(double v) { return f64_key(v); }
  __device__ static double from_s(long long v) { return key_f64(v); }
  struct K2 { long long a, b; };
  __device__ static uint4 hext(uint4 c, long long left, long long right) {
    K2 k = *reinterpret_cast<K2 *>(&c), h;
    h.a = e(e(left, k.a), k.b);
    h.b = e(e(k.a, k.b), right);
    return *reinterpret_cast<uint4 *>(&h);
  }
  __device__ static uint4 ext3(uint4 a, uint4 b, uint4 c) {
    K2 x = *reinterpret_cast<K2 *>(&a), y = *reinterpret_cast<K2 *>(&b), z = *reinterpret_cast<K2 *>(&c), r;
    r.a = e(e(x.a, y.a), z.a);
    r.b = e(e(x.b, y.b), z.b);
    return *reinterpret_cast<uint4 *>(&r);
  }
  __device__ static uint4 clamp(uint4 v, uint4 m) {
    K2 x = *reinterpret_cast<K2 *>(&v), y = *reinterpret_cast<K2 *>(&m), r;
    r.a = opp(x.a, y.a);
    r.b = opp(x.b, y.b);
    return *reinterpret_cast<uint4 *>(&r);
  }
  __device__ static long long left_word(const char *p) { return *(const long long *)(p - 8); }
  __device__ static long long right_word(const char *p) { return *(const long long *)(p + 16); }
};

// ---------------------------------------------------------------------------
// inter-CTA synchronisation with bounded waits
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}


__device__ __forceinline__ void record_status(int *status, int code) {
  atomicCAS(status, 0, code);
}

// Grid-wide barrier for a cooperative launch. Returns false (for every thread
// of the CTA) if the wait expired or an error was already recorded.
static __device__ __noinline__ bool grid_barrier(Control *ctl, int *status, unsigned nblocks,
                                                 unsigned long long limit_ns = kWaitLimitNs) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned gen = ld_acquire_u32(&ctl->bar_gen);
    __threadfence();
    unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&ctl->bar_count, 0u);
      __threadfence();
      st_release_u32(&ctl->bar_gen, gen + 1);
    } else {
      unsigned long long t0 = globaltimer_ns();
      unsigned spins = 0;
      while (ld_acquire_u32(&ctl->bar_gen) == gen) {
        if ((++spins & 63u) == 0) {
          if (globaltimer_ns() - t0 > limit_ns) {
            record_status(status, GEO_ERR_TIMEOUT);
            ok = 0;
            break;
          }
          if (*(volatile int *)status != 0) { ok = 0; break; }
        }
      }
    }
    __threadfence();
    if (*(volatile int *)status != 0) ok = 0;
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// ---------------------------------------------------------------------------
// the tile kernel
// ---------------------------------------------------------------------------

template <class E>
struct Tile {
  static constexpr int CE = E::CE;
  static constexpr int SS = E::SS;
  static constexpr int GS = E::GS;
  using G = typename E::G;

  // Load region rows [0, RH) and chunks [0, NC) (chunk 0 and NC-1 are pads)
  // of plane P at global origin (gy0, gx0) into shared buffer dst; pixels
  // outside the image get `fill`. virt: synthesise the window's virtual mask
  // (anti inside the image, ident outside) instead of reading P.
  __device__ static void load_region(char *dst, int rs, const Plane &P, int64_t H, int64_t W, int64_t gy0,
                                     int64_t gx0, int RH, int NC, bool cg, bool virt) {
    const int n = RH * NC;
    for (int i = threadIdx.x; i < n; i += kThreads) {
      const int r = i / NC, c = i - r * NC;
      const int64_t gy = gy0 + r;
      const int64_t gxc = gx0 + (int64_t)c * CE;
      uint4 out;
      auto *o = reinterpret_cast<decltype(E::ident()) *>(&out);
      const bool row_in = (gy >= 0 && gy < H);
      if (virt) {
#pragma unroll
        for (int e = 0; e < CE; ++e) {
          const int64_t gx = gxc + e;
          o[e] = (row_in && gx >= 0 && gx < W) ? E::anti() : E::ident();
        }
      } else if (row_in && gxc >= 0 && gxc + CE <= W && P.vec_ok) {
        const char *src = P.ptr + gy * P.pitch_b + gxc * GS;
        if constexpr (GS * CE == 16) {
          uint4 v = cg ? __ldcg(reinterpret_cast<const uint4 *>(src)) : __ldg(reinterpret_cast<const uint4 *>(src));
          const G *g = reinterpret_cast<const G *>(&v);
#pragma unroll
          for (int e = 0; e < CE; ++e) o[e] = E::to_s(g[e]);
        } else {  // u8: 8 pixels = 8 bytes
          uint2 v = cg ? __ldcg(reinterpret_cast<const uint2 *>(src)) : __ldg(reinterpret_cast<const uint2 *>(src));
          const G *g = reinterpret_cast<const G *>(&v);
#pragma unroll
          for (int e = 0; e < CE; ++e) o[e] = E::to_s(g[e]);
        }
      } else {
#pragma unroll
        for (int e = 0; e < CE; ++e) {
          const int64_t gx = gxc + e;
          if (row_in && gx >= 0 && gx < W) {
            const G *src = reinterpret_cast<const G *>(P.ptr + gy * P.pitch_b + gx * GS);
            o[e] = E::to_s(cg ? __ldcg(src) : __ldg(src));
          } else {
            o[e] = E::ident();
          }
        }
      }
      *reinterpret_cast<uint4 *>(dst + r * rs + c * 16) = out;
    }
  }

  // Store the tile interior (region rows [K, K+TH), pixels [K, K+TW)) from
  // shared buffer src to plane P at global tile origin (ty0, tx0). With
  // `cmp` set, also compare against plane C (the pass input) and return
  // whether any stored pixel differs.
  __device__ static bool store_interior(const char *src, int rs, const Plane &P, const Plane &C, bool cmp,
                                        int64_t H, int64_t W, int64_t ty0, int64_t tx0, int TH, int TW, int K) {
    const int NCI = TW / CE;
    const int n = TH * NCI;
    const int c0 = K / CE + 1;  // first interior chunk (after the pad)
    bool changed = false;
    for (int i = threadIdx.x; i < n; i += kThreads) {
      const int r = i / NCI, c = i - r * NCI;
      const int64_t gy = ty0 + r;
      const int64_t gxc = tx0 + (int64_t)c * CE;
      if (gy >= H || gxc >= W) continue;
      uint4 v = *reinterpret_cast<const uint4 *>(src + (K + r) * rs + (c0 + c) * 16);
      const auto *s = reinterpret_cast<const decltype(E::ident()) *>(&v);
      G g[CE];
#pragma unroll
      for (int e = 0; e < CE; ++e) g[e] = E::from_s(s[e]);
      char *dst = P.ptr + gy * P.pitch_b + gxc * GS;
      const char *cmpp = C.ptr + gy * C.pitch_b + gxc * GS;
      if (gxc + CE <= W && P.vec_ok && (!cmp || C.vec_ok)) {
        if constexpr (GS * CE == 16) {
          if (cmp) {
            uint4 old = __ldcg(reinterpret_cast<const uint4 *>(cmpp));
            uint4 nw = *reinterpret_cast<uint4 *>(g);
            changed |= (old.x != nw.x) | (old.y != nw.y) | (old.z != nw.z) | (old.w != nw.w);
          }
          __stcg(reinterpret_cast<uint4 *>(dst), *reinterpret_cast<uint4 *>(g));
        } else {
          if (cmp) {
            uint2 old = __ldcg(reinterpret_cast<const uint2 *>(cmpp));
            uint2 nw = *reinterpret_cast<uint2 *>(g);
            changed |= (old.x != nw.x) | (old.y != nw.y);
          }
          __stcg(reinterpret_cast<uint2 *>(dst), *reinterpret_cast<uint2 *>(g));
        }
      } else {
#pragma unroll
        for (int e = 0; e < CE; ++e) {
          if (gxc + e < W) {
            if (cmp) {
              G old = __ldcg(reinterpret_cast<const G *>(cmpp) + e);
              // bitwise comparison: equal values have equal bits (no NaN, no -0)
              changed |= (old != g[e]);
            }
            __stcg(reinterpret_cast<G *>(dst) + e, g[e]);
          }
        }
      }
    }
    return changed;
  }
};

// One elementary step over region rows [r0, r1) and chunks [c0, c1) (chunk
// indices include the left pad), reading shared buffer a, writing b.
template <class E, int CONN>
__device__ __forceinline__ void tile_step(const char *a, char *b, const char *m, int rs, int r0, int r1, int c0,
                                          int c1) {
  const int nc = c1 - c0, nr = r1 - r0;
  if (nc <= 0 || nr <= 0) return;
  int runs = kThreads / nc;
  if (runs < 1) runs = 1;
  if (runs > nr) runs = nr;
  const int run = (nr + runs - 1) / runs;
  runs = (nr + run - 1) / run;
  const int items = nc * runs;
  for (int it = threadIdx.x; it < items; it += kThreads) {
    const int c = c0 + it % nc;
    const int ra = r0 + (it / nc) * run;
    const int rb = min(ra + run, r1);
    const int off = c * 16;
    const char *pa = a + (ra - 1) * rs + off;
    uint4 fm = *reinterpret_cast<const uint4 *>(pa);
    uint4 hm = E::hext(fm, E::left_word(pa), E::right_word(pa));
    pa += rs;
    uint4 fc = *reinterpret_cast<const uint4 *>(pa);
    uint4 hc = E::hext(fc, E::left_word(pa), E::right_word(pa));
    const char *pm = m + ra * rs + off;
    char *pb = b + ra * rs + off;
    for (int r = ra; r < rb; ++r) {
      pa += rs;
      const uint4 fn = *reinterpret_cast<const uint4 *>(pa);
      const uint4 hn = E::hext(fn, E::left_word(pa), E::right_word(pa));
      uint4 v;
      if constexpr (CONN == 8) {
        v = E::ext3(hm, hc, hn);  // column 3-extreme of the row 3-extremes
      } else {
        v = E::ext3(fm, hc, fn);  // cross: row 3-extreme plus the pixels above and below
      }
      v = E::clamp(v, *reinterpret_cast<const uint4 *>(pm));
      *reinterpret_cast<uint4 *>(pb) = v;
      fm = fc;
      fc = fn;
      hm = hc;
      hc = hn;
      pm += rs;
      pb += rs;
    }
  }
}

template <class E, int CONN>
__global__ void __launch_bounds__(kThreads) tile_kernel(const TileLaunch L) {
  extern __shared__ __align__(16) char smem[];
  using T = Tile<E>;
  constexpr int CE = E::CE;
  const int K = L.K, TH = L.TH, TW = L.TW, rs = L.rs;
  const int RH = TH + 2 * K;
  const int NC = (TW + 2 * K) / CE + 2;  // chunks per region row, pads included
  const int buf_b = RH * rs;
  char *bufA = smem;
  char *bufB = smem + buf_b;
  char *bufM = smem + 2 * buf_b;
  const int tiles_img = L.tiles_x * L.tiles_y;
  const int ntiles = tiles_img * (L.batch > 1 ? L.batch : 1);
  const bool rec = (L.mode == MODE_REC);
  const bool virt = (L.mask.ptr == nullptr);
  // with at most one tile per CTA the mask tile stays in shared memory for
  // the whole launch; otherwise it is reloaded with every tile
  const bool mask_resident = (ntiles <= (int)gridDim.x);
  __shared__ int changed_s;

  int64_t steps_done = 0;
  int64_t steps_left = L.steps;
  for (int pass = 0;; ++pass) {
    // steps of this pass and the planes it reads and writes
    int S;
    if (!rec) {
      if (pass >= L.npasses) break;
      const int64_t base = L.steps / L.npasses, extra = L.steps % L.npasses;
      S = (int)(base + (pass < extra ? 1 : 0));
    } else {
      S = (int)(steps_left < (int64_t)K ? steps_left : (int64_t)K);
    }
    const bool to_out = rec ? (((pass + L.alias) & 1) == 0) : (((L.npasses - 1 - pass) & 1) == 0);
    const Plane dstP = to_out ? L.out : L.scratch;
    const Plane srcP = (pass == 0) ? L.marker : (to_out ? L.scratch : L.out);
    const bool src_cg = (pass > 0) || (L.marker.ptr == L.out.ptr);

    if (threadIdx.x == 0) changed_s = 0;
    bool changed = false;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int bi = t / tiles_img, tt = t - bi * tiles_img;
      const int ty = tt / L.tiles_x, tx = tt - ty * L.tiles_x;
      const Plane src = plane_of(srcP, bi), dst = plane_of(dstP, bi), mask = plane_of(L.mask, bi);
      const int64_t ty0 = (int64_t)ty * TH, tx0 = (int64_t)tx * TW;
      __syncthreads();  // previous tile's store has finished reading smem
      T::load_region(bufA, rs, src, L.H, L.W, ty0 - K, tx0 - K - CE, RH, NC, src_cg, false);
      if (!mask_resident || pass == 0)
        T::load_region(bufM, rs, mask, L.H, L.W, ty0 - K, tx0 - K - CE, RH, NC, false, virt);
      __syncthreads();
      char *a = bufA, *b = bufB;
      for (int j = 1; j <= S; ++j) {
        // rows / pixels still needed after this step: within S - j of the interior
        const int lo = K - S + j;
        const int r1 = K + TH + S - j;
        const int px1 = K + TW + S - j;
        const int c0 = lo / CE + 1;
        const int c1 = (px1 + CE - 1) / CE + 1;
        tile_step<E, CONN>(a, b, bufM, rs, lo, r1, c0, c1);
        __syncthreads();
        char *tmp = a;
        a = b;
        b = tmp;
      }
      changed |= T::store_interior(a, rs, dst, src, rec, L.H, L.W, ty0, tx0, TH, TW, K);
    }
    if (rec) {
      if (changed) changed_s = 1;
      __syncthreads();
      if (threadIdx.x == 0) {
        if (changed_s) atomicOr(&L.ctl->flags[pass % 3], 1);
        if (blockIdx.x == 0) L.ctl->flags[(pass + 1) % 3] = 0;
      }
      steps_done += S;
      steps_left -= S;
    } else if (pass == L.npasses - 1) {
      break;
    }
    if (!grid_barrier(L.ctl, L.status, gridDim.x + (L.fault ? 1u : 0u), L.wait_ns)) return;
    if (rec) {
      const int f = *(volatile int *)&L.ctl->flags[pass % 3];
      if (!f) break;  // this pass changed nothing: fixed point reached
      if (steps_left <= 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) record_status(L.status, GEO_ERR_NOT_CONVERGED);
        break;
      }
    }
  }
  if (rec && L.steps_out && blockIdx.x == 0 && threadIdx.x == 0) *L.steps_out = steps_done;
}

}  // namespace geo
