// Register-resident, temporally blocked kernel for geodesic 3x3 chains.
//
// One cooperative persistent launch per chain (Eq. 4), window (Eq. 1-2) or
// reconstruction (Eq. 5), K steps per pass on a tile plus a K-pixel halo, as
// in the shared-memory tile kernel (geo_tile.cuh); what differs is where the
// tile lives during the K steps: in registers. Chain passes synchronise
// point to point (a tile waits for the 8 tiles its halo reads to publish the
// previous pass: uint8 and rank-code chains through tagged words that carry
// the pass that wrote them, the others through per-tile epochs).
// Reconstruction of one tile per CTA (uint8, rank codes) hands over the same
// way and decides stability by a per-pass vote; otherwise its passes meet at
// a grid barrier, test a per-pass "changed" flag, and skip tiles whose 3x3
// tile neighbourhood did not change in the previous pass.
//
//   * A CTA holds a region of (32 * CW) x (NW * PH) pixels: warp w owns a
//     horizontal band of PH pixel rows, lane l owns CW adjacent columns of it.
//   * Horizontal neighbours inside a lane are in the lane's own registers;
//     the two at the lane's edges come from the adjacent lanes by __shfl.
//   * Vertical neighbours inside a warp's band are in the lane's registers;
//     the rows just above and below the band come from the adjacent warps
//     through a small shared-memory exchange, once per step (one barrier).
//   * uint8 pixels are "sliced": a 32-bit word holds the pixels of one column
//     at rows r and r + RW of the band as two 16-bit lanes, so one packed
//     max / min (f16x2 or u16x2, see GEO_RR_U8_F16) decides two pixels and no
//     byte shifts are needed except at the seam between the two halves of
//     the band (one funnel shift per column).
//   * The step itself is Section 3.1's decomposition: row 3-extreme (h),
//     column 3-extreme of h (8-conn) or of {f above, h, f below} (4-conn),
//     then the mask clamp of Eq. 3, computed in place top to bottom with the
//     h rows of the previous and next row kept in registers (the GPU
//     counterpart of Algorithm 3's two row caches).
//
// The region edges that have no neighbour (lanes 0 and 31, warps 0 and
// NW-1) read stale or identity values; that error moves inward one pixel per
// step and never reaches the tile interior, which is K pixels in.
#pragma once

#include <type_traits>

#include "geo_tile.cuh"

namespace geo {

// ---------------------------------------------------------------------------
// register-resident element policies
// ---------------------------------------------------------------------------

// Bit mask of the u8 step's min/max groups issued as f16x2 instead of
// u16x2 (1: row extremes, 2: column extremes, 4: mask clamp). The u8 values
// 0..255 in u16 lanes are, read as f16, +0 and positive subnormals whose
// order is the integer order (no flush to zero, no NaN, no -0), so both
// forms select the same lane values; on the 1024^2 1500-step chain the f16
// form measured about 3 % faster (0.78 vs 0.80 ms), whichever group uses it.
#ifndef GEO_RR_U8_F16
#define GEO_RR_U8_F16 7
#endif
// Bit mask of where policies without a one-instruction 3-extreme share the
// 2-extreme of a pair of neighbours between the two outputs that need it
// (1: row extremes of the 4-connected step, 2: column extremes of the
// 8-connected step). Measured on the 1024^2 u8 1500-step chains: the column
// sharing takes the 8-connected chain from 0.777 to 0.753 ms, the row
// sharing the 4-connected one from 0.83 to 0.80 ms; the row sharing in the
// 8-connected step made it slower (0.81 ms), so that step does not use it.
#ifndef GEO_RR_PAIRS
#define GEO_RR_PAIRS 3
#endif
// Bit mask of the u8 step's min/max groups computed by f16 arithmetic on
// the FMA pipe instead of one packed min/max on the ALU pipe (1: mask clamp,
// 2: column extremes of the band's first and last rows, 4: column extremes
// of the inner rows, 8: the shared row pairs of the column pass); each moved
// min/max costs two dependent FMA-pipe instructions instead of one ALU
// instruction. Measured on the 1024^2 u8 1500-step chains (ms, 8-conn /
// 4-conn): none 0.759 / 0.800, 1: 0.761 / 0.857, 3: 0.814, 7: 0.872,
// 15: 0.90, so the chains keep every min/max on the ALU pipe. The
// quasi-distance transform's first part, whose step also updates the keys
// of its observer on the ALU pipe, takes the clamp to the FMA pipe (1:
// 0.85 -> 0.75 ms per transform at 1024^2); its policy sets that itself.
#ifndef GEO_RR_U8_FMA
#define GEO_RR_U8_FMA 0
#endif
__device__ __forceinline__ uint32_t hmax2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("max.f16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t hmin2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("min.f16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
// relu(a - b) on both f16 lanes (one fma.relu: b * -1 + a)
__device__ __forceinline__ uint32_t hrelu_diff(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("fma.rn.relu.f16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(b), "r"(0xBC00BC00u), "r"(a));
  return r;
}
__device__ __forceinline__ uint32_t hfma2(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
// max / min of u16 lanes holding 0..255 through f16 arithmetic: read as f16
// these are +0 and positive subnormals k * 2^-24 (subnormals are kept by f16
// arithmetic), every difference of two of them is exact, so
//   max(a, b) = b + relu(a - b)   and   min(a, b) = a - relu(a - b)
// hold exactly, and no -0 arises (an exact zero sum rounds to +0).
__device__ __forceinline__ uint32_t fmax2_u8(uint32_t a, uint32_t b) {
  return hfma2(hrelu_diff(a, b), 0x3C003C00u, b);
}
__device__ __forceinline__ uint32_t fmin2_u8(uint32_t a, uint32_t b) {
  return hfma2(hrelu_diff(a, b), 0xBC00BC00u, a);
}

template <int OP, int RW_ = 4, int NW_ = 16, int FMA_ = GEO_RR_U8_FMA>
struct RU8 {
  using Wd = uint32_t;  // two u16 lanes: rows r and r + RW of one column
  using Px = uint32_t;  // one pixel value (0..255)
  using G = uint8_t;
  static constexpr int BANDS = 2, CW = 4, RW = RW_, NW = NW_, GS = 1;
  static constexpr bool PAIRS = true;  // no one-instruction 3-extreme
  static constexpr int FMA = FMA_;     // groups of GEO_RR_U8_FMA on the FMA pipe
  __device__ static Wd e2i(Wd a, Wd b) { return OP == DILATE ? umax2(a, b) : umin2(a, b); }
  __device__ static Wd e2f(Wd a, Wd b) { return OP == DILATE ? hmax2(a, b) : hmin2(a, b); }
  __device__ static Wd e2(Wd a, Wd b) { return (GEO_RR_U8_F16 & 2) ? e2f(a, b) : e2i(a, b); }
  // the same on the FMA pipe
  __device__ static Wd e2m(Wd a, Wd b) { return OP == DILATE ? fmax2_u8(a, b) : fmin2_u8(a, b); }
  __device__ static Wd ext3(Wd a, Wd b, Wd c) { return e2(e2(a, b), c); }
  // the 2-extreme of the row pass (hrow)
  __device__ static Wd e2h(Wd a, Wd b) { return (GEO_RR_U8_F16 & 1) ? e2f(a, b) : e2i(a, b); }
  __device__ static Wd ext3h(Wd a, Wd b, Wd c) { return e2h(e2h(a, b), c); }
  __device__ static Wd clamp(Wd v, Wd m) {
    if (FMA & 1) return OP == DILATE ? fmin2_u8(v, m) : fmax2_u8(v, m);
    if (GEO_RR_U8_F16 & 4) return OP == DILATE ? hmin2(v, m) : hmax2(v, m);
    return OP == DILATE ? umin2(v, m) : umax2(v, m);
  }
  // new value of a word from its neighbourhood extreme v, mask m and old value
  __device__ static Wd apply(Wd v, Wd m, Wd) { return clamp(v, m); }
  __device__ static Px ident() { return OP == DILATE ? 0u : 255u; }
  __device__ static Px anti() { return OP == DILATE ? 255u : 0u; }
  __device__ static Wd identw() { return ident() * 0x00010001u; }
  __device__ static Wd make(Px lo, Px hi) { return lo | (hi << 16); }
  __device__ static Px get(Wd w, int band) { return band ? (w >> 16) : (w & 0xffffu); }
  // word holding the pixels just above the band's two halves: the row above
  // the band (high lane of the upper warp's last word) and row RW-1 (low lane
  // of the own last word)
  __device__ static Wd up(Wd above, Wd own_last) { return __funnelshift_l(above, own_last, 16); }
  // word holding the pixels just below: row RW (high lane of own first word)
  // and the row below the band (low lane of the lower warp's first word)
  __device__ static Wd down(Wd own_first, Wd below) { return __funnelshift_r(own_first, below, 16); }
  __device__ static Px to_px(G g) { return g; }
  __device__ static G from_px(Px p) { return (G)p; }
  __device__ static uint4 pack(const Wd (&v)[CW]) { return make_uint4(v[0], v[1], v[2], v[3]); }
  __device__ static void unpack(uint4 u, Wd (&v)[CW]) {
    v[0] = u.x;
    v[1] = u.y;
    v[2] = u.z;
    v[3] = u.w;
  }
  // one lane's CW pixels of one row as loaded from global memory
  using Raw = uint32_t;
  __device__ static Raw load_raw(const char *p, bool cg) {
    return cg ? __ldcg(reinterpret_cast<const unsigned int *>(p)) : __ldg(reinterpret_cast<const unsigned int *>(p));
  }
  __device__ static void unpack_raw(Raw x, Px (&v)[CW]) {
    v[0] = x & 0xffu;
    v[1] = (x >> 8) & 0xffu;
    v[2] = (x >> 16) & 0xffu;
    v[3] = x >> 24;
  }
  // CW = 4 consecutive pixels from global memory (one 4-byte access)
  __device__ static void load_vec(const char *p, bool cg, Px (&v)[CW]) {
    const uint32_t x = cg ? __ldcg(reinterpret_cast<const unsigned int *>(p))
                          : __ldg(reinterpret_cast<const unsigned int *>(p));
    v[0] = x & 0xffu;
    v[1] = (x >> 8) & 0xffu;
    v[2] = (x >> 16) & 0xffu;
    v[3] = x >> 24;
  }
  __device__ static void store_vec(char *p, const Px (&v)[CW]) {
    __stcg(reinterpret_cast<unsigned int *>(p), v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24));
  }
  __device__ static bool differs_vec(const char *p, const Px (&v)[CW]) {
    return __ldcg(reinterpret_cast<const unsigned int *>(p)) != (v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24));
  }
};

template <int OP, int RW_ = 8, int NW_ = 16>
struct RF32 {
  using Wd = float;
  using Px = float;
  using G = float;
  static constexpr int BANDS = 1, CW = 4, RW = RW_, NW = NW_, GS = 4;
  static constexpr bool PAIRS = false;  // three-input max.f32 / min.f32
  static constexpr int FMA = 0;
  __device__ static Wd e2(Wd a, Wd b) { return OP == DILATE ? fmaxf(a, b) : fminf(a, b); }
  __device__ static Wd e2h(Wd a, Wd b) { return e2(a, b); }
  __device__ static Wd e2m(Wd a, Wd b) { return e2(a, b); }
  __device__ static Wd ext3(Wd a, Wd b, Wd c) { return OP == DILATE ? fmax3(a, b, c) : fmin3(a, b, c); }
  __device__ static Wd ext3h(Wd a, Wd b, Wd c) { return ext3(a, b, c); }
  __device__ static Wd clamp(Wd v, Wd m) { return OP == DILATE ? fminf(v, m) : fmaxf(v, m); }
  __device__ static Wd apply(Wd v, Wd m, Wd) { return clamp(v, m); }
  __device__ static Px ident() { return OP == DILATE ? -__int_as_float(0x7f800000) : __int_as_float(0x7f800000); }
  __device__ static Px anti() { return OP == DILATE ? __int_as_float(0x7f800000) : -__int_as_float(0x7f800000); }
  __device__ static Wd identw() { return ident(); }
  __device__ static Wd make(Px lo, Px) { return lo; }
  __device__ static Px get(Wd w, int) { return w; }
  __device__ static Wd up(Wd above, Wd) { return above; }
  __device__ static Wd down(Wd, Wd below) { return below; }
  __device__ static Px to_px(G g) { return g; }
  __device__ static G from_px(Px p) { return p; }
  __device__ static uint4 pack(const Wd (&v)[CW]) {
    return make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]), __float_as_uint(v[3]));
  }
  __device__ static void unpack(uint4 u, Wd (&v)[CW]) {
    v[0] = __uint_as_float(u.x);
    v[1] = __uint_as_float(u.y);
    v[2] = __uint_as_float(u.z);
    v[3] = __uint_as_float(u.w);
  }
  using Raw = float4;
  __device__ static Raw load_raw(const char *p, bool cg) {
    return cg ? __ldcg(reinterpret_cast<const float4 *>(p)) : __ldg(reinterpret_cast<const float4 *>(p));
  }
  __device__ static void unpack_raw(Raw x, Px (&v)[CW]) {
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
  }
  __device__ static void load_vec(const char *p, bool cg, Px (&v)[CW]) {
    const float4 x = cg ? __ldcg(reinterpret_cast<const float4 *>(p)) : __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
  }
  __device__ static void store_vec(char *p, const Px (&v)[CW]) {
    __stcg(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
  }
  __device__ static bool differs_vec(const char *p, const Px (&v)[CW]) {
    const uint4 o = __ldcg(reinterpret_cast<const uint4 *>(p));
    return (o.x != __float_as_uint(v[0])) | (o.y != __float_as_uint(v[1])) | (o.z != __float_as_uint(v[2])) |
           (o.w != __float_as_uint(v[3]));
  }
};

template <int OP, int RW_ = 8, int NW_ = 16>
struct RF64 {
  using Wd = long long;  // order-preserving key of the double
  using Px = long long;
  using G = double;
  static constexpr int BANDS = 1, CW = 2, RW = RW_, NW = NW_, GS = 8;
  static constexpr bool PAIRS = true;
  static constexpr int FMA = 0;
  __device__ static Wd e2(Wd a, Wd b) { return OP == DILATE ? max(a, b) : min(a, b); }
  __device__ static Wd e2h(Wd a, Wd b) { return e2(a, b); }
  __device__ static Wd e2m(Wd a, Wd b) { return e2(a, b); }
  __device__ static Wd ext3(Wd a, Wd b, Wd c) { return e2(e2(a, b), c); }
  __device__ static Wd ext3h(Wd a, Wd b, Wd c) { return ext3(a, b, c); }
  __device__ static Wd clamp(Wd v, Wd m) { return OP == DILATE ? min(v, m) : max(v, m); }
  __device__ static Wd apply(Wd v, Wd m, Wd) { return clamp(v, m); }
  __device__ static Px ident() { return OP == DILATE ? (long long)0x8000000000000000ULL : 0x7fffffffffffffffLL; }
  __device__ static Px anti() { return OP == DILATE ? 0x7fffffffffffffffLL : (long long)0x8000000000000000ULL; }
  __device__ static Wd identw() { return ident(); }
  __device__ static Wd make(Px lo, Px) { return lo; }
  __device__ static Px get(Wd w, int) { return w; }
  __device__ static Wd up(Wd above, Wd) { return above; }
  __device__ static Wd down(Wd, Wd below) { return below; }
  __device__ static Px to_px(G g) { return f64_key(g); }
  __device__ static G from_px(Px p) { return key_f64(p); }
  __device__ static uint4 pack(const Wd (&v)[CW]) {
    return make_uint4((unsigned)v[0], (unsigned)((unsigned long long)v[0] >> 32), (unsigned)v[1],
                      (unsigned)((unsigned long long)v[1] >> 32));
  }
  __device__ static void unpack(uint4 u, Wd (&v)[CW]) {
    v[0] = (long long)(((unsigned long long)u.y << 32) | u.x);
    v[1] = (long long)(((unsigned long long)u.w << 32) | u.z);
  }
  using Raw = longlong2;
  __device__ static Raw load_raw(const char *p, bool cg) {
    return cg ? __ldcg(reinterpret_cast<const longlong2 *>(p)) : __ldg(reinterpret_cast<const longlong2 *>(p));
  }
  __device__ static void unpack_raw(Raw x, Px (&v)[CW]) {
    v[0] = f64_key(__longlong_as_double(x.x));
    v[1] = f64_key(__longlong_as_double(x.y));
  }
  __device__ static void load_vec(const char *p, bool cg, Px (&v)[CW]) {
    const longlong2 x =
        cg ? __ldcg(reinterpret_cast<const longlong2 *>(p)) : __ldg(reinterpret_cast<const longlong2 *>(p));
    v[0] = f64_key(__longlong_as_double(x.x));
    v[1] = f64_key(__longlong_as_double(x.y));
  }
  __device__ static void store_vec(char *p, const Px (&v)[CW]) {
    __stcg(reinterpret_cast<longlong2 *>(p),
           make_longlong2(__double_as_longlong(key_f64(v[0])), __double_as_longlong(key_f64(v[1]))));
  }
  __device__ static bool differs_vec(const char *p, const Px (&v)[CW]) {
    const longlong2 o = __ldcg(reinterpret_cast<const longlong2 *>(p));
    return (o.x != __double_as_longlong(key_f64(v[0]))) | (o.y != __double_as_longlong(key_f64(v[1])));
  }
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---------------------------------------------------------------------------
// mbarrier helpers (shared memory, CTA scope)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
               : "memory");
}

// Wait for the phase with the given parity to complete. Gives up (returns
// false) after kWaitLimitNs so that a broken arrival count cannot hang the GPU.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  uint32_t done = 0;
  unsigned n = 0;
  unsigned long long t0 = 0;
  for (;;) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (n == 0) t0 = globaltimer_ns();
    if ((++n & 1023u) == 0 && globaltimer_ns() - t0 > kWaitLimitNs) return false;
  }
}

// 64-bit relaxed accesses at gpu scope (single-copy atomic: a tagged word is
// read whole).
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// 16-byte relaxed accesses at gpu scope: four 32-bit elements, each one
// single-copy atomic (a tagged rank-code word is read whole)
__device__ __forceinline__ uint4 ld_relaxed_v4(const unsigned *p) {
  uint4 v;
  asm volatile("ld.relaxed.gpu.global.v4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ void st_relaxed_v4(unsigned *p, uint4 v) {
  asm volatile("st.relaxed.gpu.global.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}
// a register word's bits (uint8 pairs and distances are words already)
__device__ __forceinline__ uint32_t word_bits(uint32_t x) { return x; }
__device__ __forceinline__ uint32_t word_bits(float x) { return __float_as_uint(x); }

// Policies of the single-image kernel (the batch kernel uses the defaults).
// Taller bands put more work between a warp's arrival and its wait at the
// step barrier; the host planner (rr_geom in geo_api.cu) mirrors these.
template <int OP> using SU8 = RU8<OP, GEO_RR_U8_RW, GEO_RR_U8_NW>;
template <int OP> using SF32 = RF32<OP, GEO_RR_F32_RW, GEO_RR_F32_NW>;
template <int OP> using SF64 = RF64<OP, GEO_RR_F64_RW, GEO_RR_F64_NW>;
// the autotuner's other shapes (geo_common.cuh)
template <int OP> using SU8V1 = RU8<OP, GEO_RR_U8_V1_RW, GEO_RR_U8_V1_NW>;
template <int OP> using SU8V2 = RU8<OP, GEO_RR_U8_V2_RW, GEO_RR_U8_V2_NW>;
template <int OP> using SF32V1 = RF32<OP, GEO_RR_F32_V1_RW, GEO_RR_F32_V1_NW>;
template <int OP> using SF32V2 = RF32<OP, GEO_RR_F32_V2_RW, GEO_RR_F32_V2_NW>;

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------

// Observer of the step's writes: called with (word row, column, old, new)
// for every word a step writes. The plain chains observe nothing.
struct NoObs {
  template <class Wd>
  __device__ __forceinline__ void operator()(int, int, Wd, Wd) const {}
};

template <class P>
struct RR {
  using Wd = typename P::Wd;
  using Px = typename P::Px;
  using G = typename P::G;
  static constexpr int CW = P::CW, RW = P::RW, NW = P::NW, B = P::BANDS, GS = P::GS;
  static constexpr int PH = RW * B;     // pixel rows per warp
  static constexpr int RWID = 32 * CW;  // region width in pixels
  static constexpr int RHGT = NW * PH;  // region height in pixels

  // CW pixels of global row gy starting at column gx; pixels outside the
  // image read `fill`. virt: the window's virtual mask instead of plane Q.
  __device__ static void load_px(const Plane &Q, int64_t H, int64_t W, int64_t gy, int64_t gx, bool cg, bool virt,
                                 Px (&v)[CW]) {
    const bool row_in = gy >= 0 && gy < H;
    if (virt) {
#pragma unroll
      for (int c = 0; c < CW; ++c) v[c] = (row_in && gx + c >= 0 && gx + c < W) ? P::anti() : P::ident();
      return;
    }
    if (row_in && gx >= 0 && gx + CW <= W && Q.vec_ok) {
      P::load_vec(Q.ptr + gy * Q.pitch_b + gx * GS, cg, v);
      return;
    }
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      if (row_in && gx + c >= 0 && gx + c < W) {
        const G *p = reinterpret_cast<const G *>(Q.ptr + gy * Q.pitch_b + (gx + c) * GS);
        v[c] = P::to_px(cg ? __ldcg(p) : __ldg(p));
      } else {
        v[c] = P::ident();
      }
    }
  }

  // EDGES: also batch the loads of strips that reach past the top / bottom
  // image border or lie outside it (the single-image kernel; the batch
  // kernel, which holds every element policy at once, keeps the lighter form
  // that batches only strips wholly inside the image)
  template <bool EDGES = true>
  __device__ static void load_words(const Plane &Q, int64_t H, int64_t W, int64_t gy0, int64_t gx, bool cg,
                                    bool virt, Wd (&w)[RW][CW]) {
    const bool cols_in = gx >= 0 && gx + CW <= W, cols_out = gx + CW <= 0 || gx >= W;
    if (!EDGES && !virt && Q.vec_ok && cols_in && gy0 >= 0 && gy0 + B * RW <= H) {
      typename P::Raw raw[B * RW];
#pragma unroll
      for (int i = 0; i < B * RW; ++i) raw[i] = P::load_raw(Q.ptr + (gy0 + i) * Q.pitch_b + gx * GS, cg);
#pragma unroll
      for (int r = 0; r < RW; ++r) {
        Px lo[CW], hi[CW];
        P::unpack_raw(raw[r], lo);
        if constexpr (B == 2) {
          P::unpack_raw(raw[RW + r], hi);
        } else {
#pragma unroll
          for (int c = 0; c < CW; ++c) hi[c] = lo[c];
        }
#pragma unroll
        for (int c = 0; c < CW; ++c) w[r][c] = P::make(lo[c], hi[c]);
      }
      return;
    }
    if (EDGES && !virt && Q.vec_ok && (cols_in || cols_out)) {
      // The lane's columns lie wholly inside or wholly outside the image:
      // issue the loads of every row inside before using any, so they are in
      // flight together; rows (or strips) outside the image take the identity.
      if constexpr (B == 1) {
        // one row per word: rows in chunks, which bounds the 16-byte raw
        // values live at once (f32 / f64 hold 8 rows per lane; f64 words
        // take two registers each)
        constexpr int CH = sizeof(Wd) == 8 ? 1 : 4;
        static_assert(RW % CH == 0, "word rows come in whole chunks");
#pragma unroll
        for (int r0 = 0; r0 < RW; r0 += CH) {
          typename P::Raw raw[CH];
          bool in[CH];
#pragma unroll
          for (int i = 0; i < CH; ++i) {
            const int64_t gy = gy0 + r0 + i;
            in[i] = cols_in && gy >= 0 && gy < H;
            if (in[i]) raw[i] = P::load_raw(Q.ptr + gy * Q.pitch_b + gx * GS, cg);
          }
#pragma unroll
          for (int i = 0; i < CH; ++i) {
            Px v[CW];
            P::unpack_raw(raw[i], v);
#pragma unroll
            for (int c = 0; c < CW; ++c) w[r0 + i][c] = P::make(in[i] ? v[c] : P::ident(), v[c]);
          }
        }
        return;
      } else {
        // two rows per word: every row's load first, then the words
        typename P::Raw raw[B * RW];
        bool in[B * RW];
#pragma unroll
        for (int i = 0; i < B * RW; ++i) {
          const int64_t gy = gy0 + i;
          in[i] = cols_in && gy >= 0 && gy < H;
          if (in[i]) raw[i] = P::load_raw(Q.ptr + gy * Q.pitch_b + gx * GS, cg);
        }
#pragma unroll
        for (int r = 0; r < RW; ++r) {
          Px lo[CW], hi[CW];
          P::unpack_raw(raw[r], lo);
          P::unpack_raw(raw[RW + r], hi);
#pragma unroll
          for (int c = 0; c < CW; ++c) {
            if (!in[r]) lo[c] = P::ident();
            if (!in[RW + r]) hi[c] = P::ident();
            w[r][c] = P::make(lo[c], hi[c]);
          }
        }
        return;
      }
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      Px lo[CW], hi[CW];
      load_px(Q, H, W, gy0 + r, gx, cg, virt, lo);
      if constexpr (B == 2) {
        load_px(Q, H, W, gy0 + RW + r, gx, cg, virt, hi);
      } else {
#pragma unroll
        for (int c = 0; c < CW; ++c) hi[c] = lo[c];
      }
#pragma unroll
      for (int c = 0; c < CW; ++c) w[r][c] = P::make(lo[c], hi[c]);
    }
  }

  // 2-extreme of one group of the column pass: on the FMA pipe if the
  // policy's FMA mask has the group's bit (only the u8 policy has that form)
  template <int GROUP>
  __device__ static Wd e2g(Wd a, Wd b) {
    if constexpr ((P::FMA & GROUP) != 0) return P::e2m(a, b);
    else return P::e2(a, b);
  }

  // row 3-extreme of one word row; the lane-edge neighbours come by shuffle
  template <bool PAIRED>
  __device__ static void hrow(const Wd (&row)[CW], Wd (&h)[CW]) {
    const Wd left = __shfl_up_sync(0xffffffffu, row[CW - 1], 1);
    const Wd right = __shfl_down_sync(0xffffffffu, row[0], 1);
    if constexpr (PAIRED) {
      // Without a one-instruction 3-extreme, the 2-extreme of columns
      // (2i, 2i+1) serves both outputs 2i and 2i+1: 1.5 ops per column.
      static_assert(CW % 2 == 0, "column pairs");
#pragma unroll
      for (int c = 0; c < CW; c += 2) {
        const Wd p = P::e2h(row[c], row[c + 1]);
        h[c] = P::e2h(c == 0 ? left : row[c - 1], p);
        h[c + 1] = P::e2h(p, c + 2 == CW ? right : row[c + 2]);
      }
    } else {
      h[0] = P::ext3h(left, row[0], row[1]);
#pragma unroll
      for (int c = 1; c < CW - 1; ++c) h[c] = P::ext3h(row[c - 1], row[c], row[c + 1]);
      h[CW - 1] = P::ext3h(row[CW - 2], row[CW - 1], right);
    }
  }

  // One elementary step, in place, on the lane's words. The band's boundary
  // rows go to the neighbouring warps through xb (double-buffered by step
  // parity). The CTA-wide mbarrier `bar` is split-phase: every thread
  // arrives once its rows are written, updates its inner rows (which need no
  // neighbour data), and only then waits for the phase. A phase completes
  // only when every warp has arrived for that step, and a warp arrives for
  // the next step only after its wait, so the parity of the step identifies
  // the phase and the double buffer is never overwritten before it was read. For 8-connectivity the
  // exchanged rows are the row 3-extremes h (what the neighbour needs), for
  // 4-connectivity the pixels themselves. Returns false if the wait expired.
  template <int CONN>
  __device__ static bool step(Wd (&w)[RW][CW], const Wd (&m)[RW][CW], Wd *xb, uint64_t *bar, uint32_t parity,
                              int lane, int warp) {
    NoObs none;
    return step<CONN>(w, m, xb, bar, parity, lane, warp, none);
  }

  // the same with an observer of the written words
  template <int CONN, class Obs>
  __device__ static bool step(Wd (&w)[RW][CW], const Wd (&m)[RW][CW], Wd *xb, uint64_t *bar, uint32_t parity,
                              int lane, int warp, Obs &obs) {
    static_assert(RW >= 2, "a band needs distinct first and last word rows");
    Wd *mine = xb + (size_t)(warp + 1) * 2 * RWID + lane * CW;
    const Wd *up_slot = xb + (size_t)warp * 2 * RWID + RWID + lane * CW;
    const Wd *dn_slot = xb + (size_t)(warp + 2) * 2 * RWID + lane * CW;
    Wd h[RW][CW];
    if constexpr (CONN == 8) {
      hrow<false>(w[0], h[0]);
      hrow<false>(w[RW - 1], h[RW - 1]);
      *reinterpret_cast<uint4 *>(mine) = P::pack(h[0]);
      *reinterpret_cast<uint4 *>(mine + RWID) = P::pack(h[RW - 1]);
      mbar_arrive(bar);
#pragma unroll
      for (int r = 1; r < RW - 1; ++r) hrow<false>(w[r], h[r]);
      Wd pre0[CW], preL[CW];
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        pre0[c] = e2g<8>(h[0][c], h[1][c]);
        preL[c] = e2g<8>(h[RW - 2][c], h[RW - 1][c]);
      }
#pragma unroll
      for (int r = 1; r < RW - 1; ++r)
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          Wd v;
          if constexpr (P::PAIRS && (GEO_RR_PAIRS & 2)) {
            // the same sharing down the column: pair (2i, 2i+1) of h rows
            // (pre0 for i = 0, preL for the last pair)
            static_assert(RW % 2 == 0, "row pairs");
            v = (r & 1) ? e2g<4>(r == 1 ? pre0[c] : e2g<8>(h[r - 1][c], h[r][c]), h[r + 1][c])
                        : e2g<4>(h[r - 1][c], r == RW - 2 ? preL[c] : e2g<8>(h[r][c], h[r + 1][c]));
          } else {
            v = P::ext3(h[r - 1][c], h[r][c], h[r + 1][c]);
          }
          const Wd nv = P::apply(v, m[r][c], w[r][c]);
          obs(r, c, w[r][c], nv);
          w[r][c] = nv;
        }
      const bool ok = mbar_wait(bar, parity);
      Wd ha[CW], hb[CW];
      P::unpack(*reinterpret_cast<const uint4 *>(up_slot), ha);
      P::unpack(*reinterpret_cast<const uint4 *>(dn_slot), hb);
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        // row 3-extremes of the rows just above / below the band halves
        const Wd hu = P::up(ha[c], h[RW - 1][c]);
        const Wd hd = P::down(h[0][c], hb[c]);
        const Wd n0 = P::apply(e2g<2>(pre0[c], hu), m[0][c], w[0][c]);
        const Wd nL = P::apply(e2g<2>(preL[c], hd), m[RW - 1][c], w[RW - 1][c]);
        obs(0, c, w[0][c], n0);
        obs(RW - 1, c, w[RW - 1][c], nL);
        w[0][c] = n0;
        w[RW - 1][c] = nL;
      }
      return ok;
    } else {
      *reinterpret_cast<uint4 *>(mine) = P::pack(w[0]);
      *reinterpret_cast<uint4 *>(mine + RWID) = P::pack(w[RW - 1]);
      mbar_arrive(bar);
      Wd first[CW], last[CW], pre0[CW], preL[CW];
#pragma unroll
      for (int r = 0; r < RW; ++r) hrow<P::PAIRS && (GEO_RR_PAIRS & 1)>(w[r], h[r]);
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        first[c] = w[0][c];
        last[c] = w[RW - 1][c];
        pre0[c] = P::e2(h[0][c], w[1][c]);
        preL[c] = P::e2(w[RW - 2][c], h[RW - 1][c]);
      }
      Wd fp[CW];
#pragma unroll
      for (int c = 0; c < CW; ++c) fp[c] = first[c];
#pragma unroll
      for (int r = 1; r < RW - 1; ++r) {
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          const Wd old = w[r][c];
          const Wd nv = P::apply(P::ext3(fp[c], h[r][c], w[r + 1][c]), m[r][c], old);
          obs(r, c, old, nv);
          w[r][c] = nv;
          fp[c] = old;
        }
      }
      const bool ok = mbar_wait(bar, parity);
      Wd above[CW], below[CW];
      P::unpack(*reinterpret_cast<const uint4 *>(up_slot), above);
      P::unpack(*reinterpret_cast<const uint4 *>(dn_slot), below);
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        const Wd n0 = P::apply(P::e2(pre0[c], P::up(above[c], last[c])), m[0][c], first[c]);
        const Wd nL = P::apply(P::e2(preL[c], P::down(first[c], below[c])), m[RW - 1][c], last[c]);
        obs(0, c, first[c], n0);
        obs(RW - 1, c, last[c], nL);
        w[0][c] = n0;
        w[RW - 1][c] = nL;
      }
      return ok;
    }
  }

  // store the interior part of the lane's words to D; with cmp, report
  // whether any stored pixel differs from plane C (the pass input)
  __device__ static bool store(const Wd (&w)[RW][CW], const Plane &D, const Plane &C, bool cmp, int64_t H, int64_t W,
                               int64_t ty0, int64_t tx0, int K, int TH, int TW, int lane, int warp) {
    const int X = lane * CW;
    if (X < K || X + CW > K + TW) return false;
    const int64_t gx = tx0 + (X - K);
    if (gx >= W) return false;
    const bool vec = (gx + CW <= W) && D.vec_ok && (!cmp || C.vec_ok);
    bool changed = false;
#pragma unroll
    for (int b = 0; b < B; ++b) {
#pragma unroll
      for (int r = 0; r < RW; ++r) {
        const int Y = warp * PH + b * RW + r;
        if (Y < K || Y >= K + TH) continue;
        const int64_t gy = ty0 + (Y - K);
        if (gy >= H) continue;
        Px v[CW];
#pragma unroll
        for (int c = 0; c < CW; ++c) v[c] = P::get(w[r][c], b);
        char *dp = D.ptr + gy * D.pitch_b + gx * GS;
        const char *cp = C.ptr + gy * C.pitch_b + gx * GS;
        if (vec) {
          if (cmp) changed |= P::differs_vec(cp, v);
          P::store_vec(dp, v);
        } else {
#pragma unroll
          for (int c = 0; c < CW; ++c) {
            if (gx + c < W) {
              const G g = P::from_px(v[c]);
              if (cmp) changed |= (__ldcg(reinterpret_cast<const G *>(cp) + c) != g);
              __stcg(reinterpret_cast<G *>(dp) + c, g);
            }
          }
        }
      }
    }
    return changed;
  }

  // Tagged hand-over between the passes of a uint8 chain (TileLaunch::tagged).
  // A tagged word holds one lane's CW = 4 pixels of one row in its low 32
  // bits and, in its high 32 bits, the number of passes completed when it
  // was written; the planes are zeroed before the launch. Word and tag are
  // one 64-bit access, so a reader that sees the tag it wants sees the
  // pixels written with it: the data is its own ready flag, and no release
  // fence, epoch flag or second round trip stands between a pass's stores
  // and the next pass's loads of the neighbouring tiles.
  static constexpr bool kTagged = (B == 2 && CW == 4 && sizeof(G) == 1);
  // Rank codes (the float32 policy on GEO_R32 planes): one code per 32-bit
  // word with the pass number modulo 128 in its 7 low bits, which every code
  // and both infinities (the identities) leave zero. Same bytes as a plain
  // float32 plane. The host enables it for rank-code planes only.
  static constexpr bool kTagged32 = std::is_same<Wd, float>::value && B == 1 && CW == 4;
  static constexpr bool kTaggable = kTagged || kTagged32;
  using TagW = std::conditional_t<kTagged32, unsigned, unsigned long long>;
  // tags are compared modulo kTagMask + 1 (readers want tag p while older
  // words carry p - 2 or less, so 7 bits suffice); an injected timeout waits
  // for a tag no pass writes in time
  static constexpr unsigned kTagMask = kTagged32 ? 127u : 0xffffffffu;
  static constexpr unsigned kFaultTag = kTagged32 ? 64u : (1u << 28);
  __device__ static TagW *tplane(const TileLaunch &L, int i) {
    return reinterpret_cast<TagW *>(L.tagged) + (size_t)i * L.tplane;
  }

  // Store the interior words of the lane with tag `tag`. The lane's columns
  // are whole words: K and TW are multiples of 4, so gx is. Cells past the
  // right image border hold the identity and are stored with their word.
  __device__ static void store_tagged(const Wd (&w)[RW][CW], TagW *T, int64_t tpitch, int64_t H, int64_t W,
                                      int64_t ty0, int64_t tx0, int K, int TH, int TW, unsigned tag, int lane,
                                      int warp) {
    static_assert(kTaggable, "tagged planes hold uint8 pixels or rank codes");
    const int X = lane * CW;
    if (X < K || X + CW > K + TW) return;
    const int64_t gx = tx0 + (X - K);
    if (gx >= W) return;
#pragma unroll
    for (int b = 0; b < B; ++b) {
#pragma unroll
      for (int r = 0; r < RW; ++r) {
        const int Y = warp * PH + b * RW + r;
        if (Y < K || Y >= K + TH) continue;
        const int64_t gy = ty0 + (Y - K);
        if (gy >= H) continue;
        if constexpr (kTagged32) {
          // the lane's 4 words (gx a multiple of 4; the row pitch a multiple
          // of 4 words, so columns past W up to it are written too)
          st_relaxed_v4(T + gy * tpitch + gx, make_uint4(word_bits(w[r][0]) | tag, word_bits(w[r][1]) | tag,
                                                         word_bits(w[r][2]) | tag, word_bits(w[r][3]) | tag));
        } else {
          uint32_t px = 0;
#pragma unroll
          for (int c = 0; c < CW; ++c) px |= (P::get(w[r][c], b) & 0xffu) << (8 * c);
          st_relaxed_u64(T + gy * tpitch + (gx >> 2), ((unsigned long long)tag << 32) | px);
        }
      }
    }
  }

  // Load the lane's region rows from the tagged plane T, waiting (bounded)
  // until every word inside the image carries `tag`. Rows and columns
  // outside the image take the identity. False if the wait expired.
  struct NeverStop {
    __device__ bool operator()() const { return false; }
  };
  __device__ static bool load_tagged(const TagW *T, int64_t tpitch, int64_t H, int64_t W, int64_t gy0, int64_t gx,
                                     unsigned tag, unsigned long long limit_ns, Wd (&w)[RW][CW]) {
    NeverStop never;
    return load_tagged_or_stop(T, tpitch, H, W, gy0, gx, tag, limit_ns, w, never) == 1;
  }

  // The same, but while waiting the lane also asks `stop` now and then; when
  // it answers true the lane gives up. 1 = loaded, 0 = the wait expired, 2 =
  // stopped. A stopped lane's interior cells (those its tile stores) hold
  // its tile's own words of the previous pass: uint8 keeps w as it was (the
  // registers that were stored), rank codes load in place, and a tile's own
  // words are visible to it before the next pass (a CTA barrier stands
  // between its stores and its loads), so they arrive with the tag wanted.
  template <class Stop>
  __device__ static int load_tagged_or_stop(const TagW *T, int64_t tpitch, int64_t H, int64_t W, int64_t gy0,
                                            int64_t gx, unsigned tag, unsigned long long limit_ns, Wd (&w)[RW][CW],
                                            const Stop &stop) {
    static_assert(kTaggable, "tagged planes hold uint8 pixels or rank codes");
    if constexpr (kTagged32) {
      return load_tagged32(T, tpitch, H, W, gy0, gx, tag, limit_ns, w, stop);
    } else {
      return load_tagged64(T, tpitch, H, W, gy0, gx, tag, limit_ns, w, stop);
    }
  }

  // rank codes: the lane's 4 words of each of its rows in one 16-byte load,
  // straight into w (no second copy of the region in registers), the tags
  // checked per word and then cleared
  template <class Stop>
  __device__ static int load_tagged32(const unsigned *T, int64_t tpitch, int64_t H, int64_t W, int64_t gy0,
                                      int64_t gx, unsigned tag, unsigned long long limit_ns, Wd (&w)[RW][CW],
                                      const Stop &stop) {
    constexpr int NR = RW;  // one band
    const bool cols = gx >= 0 && gx < W;
    const unsigned *col = T + (cols ? gx : 0);
    unsigned in = 0;
    auto fetch = [&](int i) {
      const uint4 v = ld_relaxed_v4(col + (gy0 + i) * tpitch);
      w[i][0] = __uint_as_float(v.x);
      w[i][1] = __uint_as_float(v.y);
      w[i][2] = __uint_as_float(v.z);
      w[i][3] = __uint_as_float(v.w);
    };
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const int64_t gy = gy0 + i;
      if (cols && gy >= 0 && gy < H) {
        fetch(i);
        in |= 1u << i;
      }
    }
    int res = 1;
    unsigned n = 0;
    unsigned long long t0 = 0;
    for (;;) {
      unsigned miss = 0;
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        const uint32_t d = (word_bits(w[i][0]) ^ tag) | (word_bits(w[i][1]) ^ tag) | (word_bits(w[i][2]) ^ tag) |
                           (word_bits(w[i][3]) ^ tag);
        if (((in >> i) & 1u) && (d & kTagMask) != 0u) miss |= 1u << i;
      }
      if (!miss) break;
      if (n == 0) t0 = globaltimer_ns();
      if ((++n & 15u) == 0) {
        if (stop()) {
          res = 2;
          break;
        }
        if (globaltimer_ns() - t0 > limit_ns) {
          res = 0;
          break;
        }
      }
#pragma unroll
      for (int i = 0; i < NR; ++i)
        if ((miss >> i) & 1u) fetch(i);
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        const bool cin = ((in >> r) & 1u) && gx + c < W;
        w[r][c] = cin ? __uint_as_float(word_bits(w[r][c]) & ~kTagMask) : P::ident();
      }
    }
    return res;
  }

  // uint8: 64-bit words of 4 pixels and a 32-bit tag, loaded into a copy so
  // that a stopped lane keeps w
  template <class Stop>
  __device__ static int load_tagged64(const unsigned long long *T, int64_t tpitch, int64_t H, int64_t W, int64_t gy0,
                                      int64_t gx, unsigned tag, unsigned long long limit_ns, Wd (&w)[RW][CW],
                                      const Stop &stop) {
    constexpr int NR = B * RW;
    const bool cols = gx >= 0 && gx < W;
    const unsigned long long *col = T + (cols ? (gx >> 2) : 0);
    unsigned long long raw[NR];
    unsigned in = 0;
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const int64_t gy = gy0 + i;
      raw[i] = 0;
      if (cols && gy >= 0 && gy < H) {
        raw[i] = ld_relaxed_u64(col + gy * tpitch);
        in |= 1u << i;
      }
    }
    bool ok = true;
    unsigned n = 0;
    unsigned long long t0 = 0;
    for (;;) {
      unsigned miss = 0;
#pragma unroll
      for (int i = 0; i < NR; ++i)
        if (((in >> i) & 1u) && (unsigned)(raw[i] >> 32) != tag) miss |= 1u << i;
      if (!miss) break;
      if (n == 0) t0 = globaltimer_ns();
      if ((++n & 15u) == 0) {
        if (stop()) return 2;
        if (globaltimer_ns() - t0 > limit_ns) {
          ok = false;
          break;
        }
      }
#pragma unroll
      for (int i = 0; i < NR; ++i)
        if ((miss >> i) & 1u) raw[i] = ld_relaxed_u64(col + (gy0 + i) * tpitch);
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      Px lo[CW], hi[CW];
      P::unpack_raw((uint32_t)raw[r], lo);
      P::unpack_raw((uint32_t)raw[RW + r], hi);
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        const bool cin = gx + c < W;
        if (!((in >> r) & 1u) || !cin) lo[c] = P::ident();
        if (!((in >> (RW + r)) & 1u) || !cin) hi[c] = P::ident();
        w[r][c] = P::make(lo[c], hi[c]);
      }
    }
    return ok ? 1 : 0;
  }
};

// Wait until every tile of the 3x3 tile neighbourhood of (ty, tx) has
// published epoch >= want. Called by all lanes of one warp: lane k < 9 polls
// neighbour k, so the eight acquire loads are in flight together instead of
// one after another. Bounded; false (on every lane) if a wait expired.
__device__ __forceinline__ bool wait_neighbours(const int *epoch, int ty, int tx, int tiles_y, int tiles_x,
                                                int want, int lane, unsigned long long limit_ns) {
  bool ok = true;
  if (lane < 9 && lane != 4) {
    const int ny = ty + lane / 3 - 1, nx = tx + lane % 3 - 1;
    if (ny >= 0 && ny < tiles_y && nx >= 0 && nx < tiles_x) {
      const unsigned *f = reinterpret_cast<const unsigned *>(epoch) + ny * tiles_x + nx;
      const unsigned long long t0 = globaltimer_ns();
      unsigned spins = 0;
      while ((int)ld_acquire_u32(f) < want) {
        if ((++spins & 255u) == 0 && globaltimer_ns() - t0 > limit_ns) {
          ok = false;
          break;
        }
      }
    }
  }
  // the acquire loads, followed by the caller's CTA barrier, order every
  // thread's later loads of the neighbours' tiles after their stores
  return __all_sync(0xffffffffu, ok);
}

// Whether any tile of the 3x3 tile neighbourhood of (ty, tx) has a non-zero
// flag (flags of one image, the previous pass).
__device__ __forceinline__ int any_neighbour_changed(const int *flags, int ty, int tx, int tiles_y, int tiles_x) {
  for (int dy = -1; dy <= 1; ++dy) {
    const int ny = ty + dy;
    if (ny < 0 || ny >= tiles_y) continue;
    for (int dx = -1; dx <= 1; ++dx) {
      const int nx = tx + dx;
      if (nx < 0 || nx >= tiles_x) continue;
      if (__ldcg(flags + ny * tiles_x + nx)) return 1;
    }
  }
  return 0;
}

// ---------------------------------------------------------------------------
// reconstruction with tagged planes (uint8 or rank codes, one tile per CTA)
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// The outcome of the passes from `chk` on, before pass `upto`: the first
// pass whose last step changed no pixel anywhere (the image is then a fixed
// point), -1 while none is known, -2 once a tile has given up. chk advances
// over the passes known to have changed something.
__device__ __forceinline__ int rec_poll(const TileLaunch &L, int &chk, int upto) {
  if (ld_acquire_u32(reinterpret_cast<const unsigned *>(L.rec_abort))) return -2;
  while (chk < upto) {
    const unsigned r = ld_acquire_u32(L.rec_res + (chk % kRecRing));
    if ((r >> 2) != (unsigned)(chk + 1)) return -1;  // not decided yet
    if ((r & 3u) == 2u) return chk;
    ++chk;
  }
  return -1;
}

// Stop test of a tile waiting for its neighbours' words: the fixed point is
// known, or some tile gave up.
struct RecStop {
  const TileLaunch *L;
  int chk;
  __device__ bool operator()() const {
    int c = chk;
    return rec_poll(*L, c, 0x7fffffff) != -1;
  }
};

// Observer of a pass's last step: whether any pixel of the tile's interior
// (and inside the image) changed. colmask: the lane's interior columns (bit
// c); rowmask[r]: the interior rows among the two u16 lanes of word row r
// (uint8), or bit r of rowmask[0] for an interior word row (rank codes).
template <class P>
struct InteriorChange {
  static constexpr int NM = P::BANDS == 2 ? P::RW : 1;
  uint32_t colmask;
  uint32_t rowmask[NM];  // one band (rank codes): bit r of rowmask[0] for word row r
  bool changed;
  template <class Wd>
  __device__ __forceinline__ void operator()(int r, int c, Wd old, Wd nv) {
    if constexpr (P::BANDS == 2) {
      if ((colmask >> c) & 1u) changed |= ((word_bits(old) ^ word_bits(nv)) & rowmask[r]) != 0u;
    } else {
      if (((colmask >> c) & (rowmask[0] >> r) & 1u) != 0u) changed |= word_bits(old) != word_bits(nv);
    }
  }
};

template <class P>
constexpr size_t rr_smem_bytes() {
  return sizeof(typename P::Wd) * 2 * (P::NW + 2) * 2 * 32 * P::CW;
}

// TAG: the variant whose chains hand the passes over in tagged planes
// (uint8 or rank codes, one tile per CTA; TileLaunch::tagged). A separate
// instantiation, so that the plain kernel's code is not touched by it.
// Blocks of 8 warps or fewer (the smaller shape variants) are bounded to
// 128 registers a thread, so that two of them fit on one SM.
template <class P, int CONN, bool TAG = false>
__global__ void __launch_bounds__(P::NW * 32, P::NW <= 8 ? 2 : 1) rr_kernel(const TileLaunch L) {
  using R = RR<P>;
  static_assert(!TAG || R::kTaggable, "tagged planes hold uint8 pixels or rank codes");
  using Wd = typename P::Wd;
  constexpr int CW = R::CW, RW = R::RW, NW = R::NW, PH = R::PH, RWID = R::RWID;
  // boundary-row exchange buffer [parity][warp slot][top/bottom][column], in
  // dynamic shared memory (rr_smem_bytes) because with many warps it exceeds
  // the 48 KB of static shared memory
  extern __shared__ __align__(16) char rr_dyn[];
  Wd(*xbuf)[NW + 2][2][RWID] = reinterpret_cast<Wd(*)[NW + 2][2][RWID]>(rr_dyn);
  __shared__ int changed_s, active_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int K = L.K, TH = L.TH, TW = L.TW;
  const int tiles_img = L.tiles_x * L.tiles_y;
  const int ntiles = tiles_img * (L.batch > 1 ? L.batch : 1);
  const bool rec = (L.mode == MODE_REC);
  const bool virt = (L.mask.ptr == nullptr);
  const bool mask_resident = (ntiles <= (int)gridDim.x);
  // tagged hand-over between passes (one tile per CTA, uint8 or rank codes):
  // chains, and reconstruction in its own loop below
  const bool tagged = TAG && L.tagged != nullptr && mask_resident;

  __shared__ __align__(8) uint64_t xbar;  // split-phase step barrier of the whole CTA
  if (threadIdx.x == 0) mbar_init(&xbar, NW * 32);
  // the slots above warp 0 and below warp NW-1 hold the identity
  for (int i = threadIdx.x; i < 2 * 2 * RWID; i += NW * 32) {
    const int par = i / (2 * RWID), rest = i % (2 * RWID);
    (&xbuf[par][0][0][0])[rest] = P::identw();
    (&xbuf[par][NW + 1][0][0])[rest] = P::identw();
  }
  __syncthreads();

  Wd w[RW][CW], m[RW][CW];
  int64_t steps_left = L.steps, steps_done = 0;
  int parity = 0;  // parity of the steps done by this CTA: exchange buffer and barrier phase

  if constexpr (TAG) {
    if (rec && tagged) {
      // Reconstruction with the tagged hand-over: no grid barrier. After each
      // pass a tile reports whether the pass's last step changed a pixel of
      // its interior (one vote word per pass, in a ring); the last tile to
      // report a pass publishes its outcome. A step that changes nothing
      // anywhere means the image is a fixed point (the step is a function of
      // the image), so the first pass whose last step changed nothing is the
      // last one needed. Tiles go on to the next passes meanwhile (at most one
      // pass ahead of any neighbour, as in a chain) and stop at the start of
      // a pass, or while waiting for a neighbour's words, once they know that
      // outcome; the registers then hold a later pass's interior, which is the
      // same fixed point, and go to out.
      __shared__ int rs_stop, rs_chk;
      const int t = blockIdx.x;
      if (t < ntiles) {
        const int ty = t / L.tiles_x, tx = t - ty * L.tiles_x;
        const int64_t ty0 = (int64_t)ty * TH, tx0 = (int64_t)tx * TW;
        const int64_t gy0 = ty0 - K + warp * PH;
        const int64_t gx = tx0 - K + lane * CW;
        R::load_words(L.mask, L.H, L.W, gy0, gx, false, virt, m);
        R::load_words(L.marker, L.H, L.W, gy0, gx, L.marker.ptr == L.out.ptr, false, w);
        InteriorChange<P> ic;
        ic.colmask = 0;
        ic.changed = false;
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          const int X = lane * CW + c;
          if (X >= K && X < K + TW && tx0 + (X - K) < L.W) ic.colmask |= 1u << c;
        }
        if constexpr (R::B == 2) {
#pragma unroll
          for (int r = 0; r < RW; ++r) {
            uint32_t rm = 0;
#pragma unroll
            for (int b = 0; b < R::B; ++b) {
              const int Y = warp * PH + b * RW + r;
              if (Y >= K && Y < K + TH && ty0 + (Y - K) < L.H) rm |= 0xffffu << (16 * b);
            }
            ic.rowmask[r] = rm;
          }
        } else {
          ic.rowmask[0] = 0;
#pragma unroll
          for (int r = 0; r < RW; ++r) {
            const int Y = warp * PH + r;
            if (Y >= K && Y < K + TH && ty0 + (Y - K) < L.H) ic.rowmask[0] |= 1u << r;
          }
        }
        int chk = 0, stop_pass = -1;
        bool aborted = false;
        int64_t left = L.steps, done = 0;
        // thread 0's vote on the previous pass: the pass's word before its
        // own add (tiles done in the low 16 bits, tiles changed in the high
        // ones), read only after the next pass's loads, so that the atomic's
        // round trip overlaps them; the last tile of a pass publishes its
        // outcome then
        unsigned vote_old = 0, vote_mine = 0;
        int vote_pass = -1;
        auto settle_vote = [&]() {
          if (vote_pass >= 0 && (vote_old & 0xffffu) == (unsigned)(ntiles - 1)) {
            const unsigned slot = (unsigned)(vote_pass % kRecRing);
            const bool changed = (vote_old >> 16) + vote_mine > 0u;
            L.rec_done[slot] = 0;  // free for pass vote_pass + kRecRing
            st_release_u32(L.rec_res + slot, ((unsigned)(vote_pass + 1) << 2) | (changed ? 1u : 2u));
          }
          vote_pass = -1;
        };
        for (int q = 0;; ++q) {
          if (q > 0) {
            // the outcome of pass chk and the abort flag, read by thread 0
            // now and looked at after this pass's loads
            unsigned pre_res = 0, pre_abort = 0;
            if (threadIdx.x == 0) {
              pre_res = ld_relaxed_u32(L.rec_res + (chk % kRecRing));
              pre_abort = ld_relaxed_u32(reinterpret_cast<const unsigned *>(L.rec_abort));
              rs_chk = chk;
            }
            __syncthreads();
            // this pass's region: the previous pass's words of this tile and
            // its neighbours, unless the fixed point becomes known meanwhile
            RecStop stop{&L, rs_chk};
            const unsigned want = ((unsigned)q + (L.fault ? R::kFaultTag : 0u)) & R::kTagMask;
            const int lr =
                R::load_tagged_or_stop(R::tplane(L, (q - 1) & 1), L.tpitch, L.H, L.W, gy0, gx, want, L.wait_ns, w, stop);
            const int failed = __syncthreads_or(lr == 0);
            const int stopped = __syncthreads_or(lr == 2);
            if (threadIdx.x == 0) {
              settle_vote();
              int sp = -1;
              if (pre_abort) {
                sp = -2;
              } else if ((pre_res >> 2) == (unsigned)(chk + 1)) {
                if ((pre_res & 3u) == 2u) sp = chk;
                else ++chk;
              }
              if (stopped && sp == -1) sp = rec_poll(L, chk, 0x7fffffff);  // a lane saw the outcome
              rs_stop = sp;
            }
            __syncthreads();
            if (failed) {
              if (threadIdx.x == 0) {
                record_status(L.status, GEO_ERR_TIMEOUT);
                atomicExch(L.rec_abort, 1);
              }
              aborted = true;
              break;
            }
            const int sp = rs_stop;
            if (sp >= 0) {
              stop_pass = sp;
              break;
            }
            if (sp == -2) {
              aborted = true;
              break;
            }
          }
          const int S = (int)(left < K ? left : K);
          bool ok = true;
          ic.changed = false;
          for (int j = 0; j < S; ++j) {
            if (j == S - 1) ok &= R::template step<CONN>(w, m, &xbuf[parity][0][0][0], &xbar, parity, lane, warp, ic);
            else ok &= R::template step<CONN>(w, m, &xbuf[parity][0][0][0], &xbar, parity, lane, warp);
            parity ^= 1;
          }
          const int tile_changed = __syncthreads_or(ic.changed ? 1 : 0);
          if (__syncthreads_or(ok ? 0 : 1)) {
            if (threadIdx.x == 0) {
              record_status(L.status, GEO_ERR_TIMEOUT);
              atomicExch(L.rec_abort, 1);
            }
            aborted = true;
            break;
          }
          R::store_tagged(w, R::tplane(L, q & 1), L.tpitch, L.H, L.W, ty0, tx0, K, TH, TW,
                          (unsigned)(q + 1) & R::kTagMask, lane, warp);
          left -= S;
          done += S;
          if (threadIdx.x == 0) {
            // acq_rel: the last tile's read of the word synchronises with
            // every tile's vote on it (and what came before the votes)
            vote_mine = tile_changed ? 1u : 0u;
            vote_old = atom_add_acq_rel_u32(reinterpret_cast<unsigned *>(L.rec_done + q % kRecRing),
                                            1u | (vote_mine << 16));
            vote_pass = q;
          }
          if (left <= 0) {
            // the step cap: this pass's outcome decides between a fixed point
            // and GEO_ERR_NOT_CONVERGED (every tile reaches the cap together)
            if (threadIdx.x == 0) {
              settle_vote();
              int sp = -1;
              const unsigned long long t0 = globaltimer_ns();
              unsigned spins = 0;
              while ((sp = rec_poll(L, chk, q + 1)) == -1 && chk <= q) {
                if ((++spins & 255u) == 0 && globaltimer_ns() - t0 > L.wait_ns) {
                  record_status(L.status, GEO_ERR_TIMEOUT);
                  atomicExch(L.rec_abort, 1);
                  sp = -2;
                  break;
                }
              }
              rs_stop = sp;
            }
            __syncthreads();
            const int sp = rs_stop;
            if (sp >= 0) stop_pass = sp;
            else if (sp == -2) aborted = true;
            else if (t == 0 && threadIdx.x == 0) record_status(L.status, GEO_ERR_NOT_CONVERGED);
            break;
          }
        }
        // every outcome this tile acted on was published with a release; the
        // fence orders the reads that saw them before the stores to out
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        if (!aborted) R::store(w, L.out, L.out, false, L.H, L.W, ty0, tx0, K, TH, TW, lane, warp);
        if (L.steps_out && t == 0 && threadIdx.x == 0) {
          const int64_t applied = (int64_t)(stop_pass + 1) * K;
          *L.steps_out = stop_pass >= 0 ? (applied < L.steps ? applied : L.steps) : done;
        }
      }
      return;
    }
  }
  for (int pass = 0;; ++pass) {
    int S;
    if (!rec) {
      if (pass >= L.npasses) break;
      const int64_t base = L.steps / L.npasses, extra = L.steps % L.npasses;
      S = (int)(base + (pass < extra ? 1 : 0));
    } else {
      // one tile covering one image: no halo exchange, test every kSoloRecSteps steps
      const int64_t Kp = (ntiles == 1) ? kSoloRecSteps : K;
      S = (int)(steps_left < Kp ? steps_left : Kp);
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
      const int64_t gy0 = ty0 - K + warp * PH;
      const int64_t gx = tx0 - K + lane * CW;
      if (!rec && pass > 0 && !tagged) {
        // chains synchronise point to point: the tiles whose interiors this
        // tile's halo reads must have finished the previous pass (which also
        // means they are done reading the buffer this pass overwrites)
        if (warp == 0 &&
            !wait_neighbours(L.epoch + (size_t)bi * tiles_img, ty, tx, L.tiles_y, L.tiles_x,
                             L.fault ? pass + (1 << 28) : pass, lane, L.wait_ns) &&
            lane == 0)
          record_status(L.status, GEO_ERR_TIMEOUT);
        __syncthreads();
      }
      int steps_here = S;
      if (rec && pass >= 1) {
        // Work-efficient reconstruction: if no tile of this tile's 3x3 tile
        // neighbourhood changed in the previous pass, this tile's region is
        // what it was one pass ago, so this pass cannot change it either
        // (the chain is monotone from its first step on). From pass 2 on both
        // ping-pong buffers already hold its current interior and it is
        // skipped; in pass 1 the second buffer is still unwritten, so the
        // interior is copied without steps.
        const int *prev = L.tchg + (size_t)((pass - 1) & 1) * ntiles + (size_t)bi * tiles_img;
        if (threadIdx.x == 0) active_s = any_neighbour_changed(prev, ty, tx, L.tiles_y, L.tiles_x);
        __syncthreads();
        if (!active_s) {
          if (threadIdx.x == 0) L.tchg[(size_t)(pass & 1) * ntiles + t] = 0;
          if (pass >= 2) continue;
          steps_here = 0;
        }
      }
      bool loaded = false;
      if constexpr (TAG) {
        if (tagged && pass > 0) {
          // the previous pass's words: from this tile's own threads (its
          // interior) and from the 8 neighbouring tiles (the halo)
          const unsigned want = ((unsigned)pass + (L.fault ? R::kFaultTag : 0u)) & R::kTagMask;
          if (!R::load_tagged(R::tplane(L, (pass - 1) & 1), L.tpitch, L.H, L.W, gy0, gx, want, L.wait_ns, w))
            record_status(L.status, GEO_ERR_TIMEOUT);
          loaded = true;
        }
      }
      if (!loaded) R::load_words(src, L.H, L.W, gy0, gx, src_cg, false, w);
      if (!mask_resident || pass == 0) R::load_words(mask, L.H, L.W, gy0, gx, false, virt, m);
      // Tagged hand-over, write-after-read: no fence stands between this
      // pass's loads and its stores. A tile overwrites a plane word that a
      // neighbour reads (tag p - 1 replaced by p + 1) only in a pass whose
      // loads saw the neighbour's words of tag p, and the neighbour stored
      // those only after every load of its own pass p - 1 had returned the
      // tag it waited for: each tile's stores depend (through its bounded
      // tag check) on its loads. An overwrite that reached the neighbour's
      // load first would return tag p + 1, fail that check and so prevent
      // the very stores it depends on: a causal cycle, excluded by the PTX
      // memory model's no-thin-air axiom. The plain first and last passes
      // (marker in, out written, possibly in place) are ordered the same
      // way, through at least one tagged pass between them. Were such an
      // overwrite ever observed, the reader would see a tag it does not
      // want and its bounded wait would report GEO_ERR_TIMEOUT instead of
      // using the pixels. A fence.acq_rel.gpu here held each warp about
      // 1100 SM clocks per pass (the bench's 1024^2 u8 1500-step chain:
      // 0.721 ms with it, 0.707 ms without).
      bool ok = true;
      for (int j = 0; j < steps_here; ++j) {
        ok &= R::template step<CONN>(w, m, &xbuf[parity][0][0][0], &xbar, parity, lane, warp);
        parity ^= 1;
      }
      if (!ok) record_status(L.status, GEO_ERR_TIMEOUT);
      bool stored = false;
      if constexpr (TAG) {
        if (tagged && pass + 1 < L.npasses) {
          R::store_tagged(w, R::tplane(L, pass & 1), L.tpitch, L.H, L.W, ty0, tx0, K, TH, TW,
                          (unsigned)(pass + 1) & R::kTagMask, lane, warp);
          stored = true;
        }
      }
      const bool tile_changed =
          stored ? false : R::store(w, dst, src, rec, L.H, L.W, ty0, tx0, K, TH, TW, lane, warp);
      changed |= tile_changed;
      if (rec) {
        const int any = __syncthreads_or(tile_changed ? 1 : 0);
        if (threadIdx.x == 0) L.tchg[(size_t)(pass & 1) * ntiles + t] = any;
      }
      if (!rec && pass + 1 < L.npasses && !tagged) {
        // every thread's stores of this tile happen before the barrier, and
        // the barrier before thread 0's release store, so the release (which
        // is cumulative) publishes the whole tile at gpu scope
        __syncthreads();
        if (threadIdx.x == 0) st_release_u32(reinterpret_cast<unsigned *>(L.epoch) + t, (unsigned)(pass + 1));
      }
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
    } else {
      if (pass == L.npasses - 1) break;
      continue;  // no grid barrier between chain passes (every wait is bounded)
    }
    if (!grid_barrier(L.ctl, L.status, gridDim.x + (L.fault ? 1u : 0u), L.wait_ns)) return;
    if (rec) {
      const int f = *(volatile int *)&L.ctl->flags[pass % 3];
      if (!f) break;
      if (steps_left <= 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) record_status(L.status, GEO_ERR_NOT_CONVERGED);
        break;
      }
    }
  }
  if (rec && L.steps_out && blockIdx.x == 0 && threadIdx.x == 0) *L.steps_out = steps_done;
}

}  // namespace geo
