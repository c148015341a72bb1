// Shared device/host definitions of the geomorph CUDA library (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/geomorph.h"

namespace geo {

enum Op : int { DILATE = 0, ERODE = 1 };
enum Mode : int { MODE_CHAIN = 0, MODE_REC = 1 };

// Internal element type next to geo_dtype: int32 distances held as u16
// lanes (the eta iteration of the quasi-distance transform, geo_qdt.cu).
constexpr int GEO_D32 = 3;
// Internal element type of the float64 rank transform (geo_rank.cu): float32
// planes whose values are rank codes, non-negative finite floats whose 7 low
// bits are zero (rank_code). The float32 kernel computes on them unchanged;
// the 7 free bits let its passes hand over in tagged 32-bit words.
constexpr int GEO_R32 = 4;
// rank r <-> its code's bit pattern: (r + 2^16) << 7 is a normal positive
// float (no subnormals) below +inf for every r < kMaxRankCodes
constexpr uint32_t kRankCodeBase = 1u << 16;
constexpr int64_t kMaxRankCodes = (int64_t)(0x7f800000u >> 7) - kRankCodeBase;

constexpr int kThreads = 256;  // threads per CTA of the tile kernels

// A spin on another CTA gives up after this long and records GEO_ERR_TIMEOUT
// (TileLaunch::wait_ns; GEOMORPH_FAULT=timeout shortens it to kFaultWaitNs).
constexpr unsigned long long kWaitLimitNs = 4000000000ULL;  // 4 s
constexpr unsigned long long kFaultWaitNs = 20000000ULL;    // 20 ms

// Band height (word rows per warp) and warps per CTA of the single-image
// register-resident kernel, per element type.
#ifndef GEO_RR_U8_RW
#define GEO_RR_U8_RW 4
#define GEO_RR_U8_NW 16
#endif
#ifndef GEO_RR_F32_RW
#define GEO_RR_F32_RW 8
#define GEO_RR_F32_NW 16
#endif
#ifndef GEO_RR_F64_RW
#define GEO_RR_F64_RW 8
#define GEO_RR_F64_NW 16
#endif

// Pre-built shapes of the register-resident kernel that the autotuner can
// choose among (variant 0 is the default above). uint8: 128x64 pixels with
// 8 warps and 128x96 with 12 warps; float32: 128x64 with 8 warps of 8 rows
// and 128x64 with 16 warps of 4 rows. Smaller regions give an image more
// tiles, which pays when its tiles alone would leave SMs idle.
constexpr int kRRVariants = 3;
#define GEO_RR_U8_V1_RW 4
#define GEO_RR_U8_V1_NW 8
#define GEO_RR_U8_V2_RW 4
#define GEO_RR_U8_V2_NW 12
#define GEO_RR_F32_V1_RW 8
#define GEO_RR_F32_V1_NW 8
#define GEO_RR_F32_V2_RW 4
#define GEO_RR_F32_V2_NW 16

// One image operand of a pass: base pointer, row stride in bytes, and
// whether 16-byte vector access is legal (base and stride 16-byte aligned).
struct Plane {
  char *ptr;
  int64_t pitch_b;
  int vec_ok;
  int64_t bstride;  // bytes from one image of a batch to the next
};

__host__ __device__ inline Plane plane_of(const Plane &P, int b) {
  Plane q = P;
  if (q.ptr) q.ptr += (int64_t)b * P.bstride;
  return q;
}

// Inter-CTA control words, zeroed by the host before each launch.
struct Control {
  unsigned int bar_count;  // grid barrier arrivals
  unsigned int bar_gen;    // grid barrier generation
  int flags[3];            // per-pass "changed" flags (rotating)
  int pad;
};

struct TileLaunch {
  Plane marker;   // input of pass 0
  Plane mask;     // mask (ptr == nullptr: unmasked window, virtual mask)
  Plane out;      // caller's output
  Plane scratch;  // library scratch (ping-pong partner of out)
  int64_t H, W;
  int TH, TW, K;          // tile interior (px) and halo (px)
  int tiles_x, tiles_y;
  int rs;                 // shared-memory row stride in bytes
  int mode;               // MODE_CHAIN or MODE_REC
  int npasses;            // chain: number of passes
  int64_t steps;          // chain: total steps; rec: max steps
  int alias;              // rec: 1 if out aliases marker
  Control *ctl;
  int *status;            // per-device sticky status word
  int64_t *steps_out;     // rec: optional device pointer
  int batch;              // images of equal shape, one after another (<= 1: one image)
  int *epoch;             // register kernel, chains: per tile, passes completed
  int *tchg;              // register kernel, reconstruction: [2][tiles] changed flags per pass
  unsigned long long wait_ns;  // limit of every wait on another CTA
  int fault;              // injected failure (GEOMORPH_FAULT=timeout): the waits on other CTAs
                          // wait for something that never happens, expire and report GEO_ERR_TIMEOUT
  // register kernel, uint8 and rank-code chains with one tile per CTA: the
  // passes hand their results over in two planes of tagged words instead of
  // plain planes plus tile epochs; nullptr: off. uint8: 64-bit words of 4
  // pixels + the number of the pass that wrote them; rank codes: 32-bit
  // words of one code with that number modulo 128 in its 7 low bits
  unsigned long long *tagged;
  int64_t tpitch, tplane;  // words per row / per plane of `tagged` (in the element's tagged words)
  // register kernel, uint8 and rank-code reconstruction with tagged planes (one tile per
  // CTA): per-pass words in a ring of kRecRing slots, zeroed with the control
  // words: the votes (tiles done with the pass in the low 16 bits, tiles
  // whose interior changed in the pass's last step in the high 16), the
  // pass's outcome ((pass + 1) << 2 | 1 changed, | 2 unchanged), and a flag
  // set by a tile whose wait expired
  int *rec_done;
  unsigned *rec_res;
  int *rec_abort;
};

// Ring of per-pass reconstruction counters: a tile is at most one pass ahead
// of each neighbour, so no two tiles are more than (tiles - 1) passes apart
// (at most 2 CTAs per SM, 304 tiles on 152 SMs), and a slot is reused only
// after every tile has finished the pass that used it before.
constexpr int kRecRing = 512;

// Passes of a chain of `steps` with halo K; K = 0 for a single-tile plan of
// the register kernel. When one tile covers the image (one image, one tile),
// every cell of its region outside the interior lies outside the image and
// stays the identity step after step (the mask clamp pins it), and there is
// no neighbouring tile to exchange with: the steps need no pass boundaries
// at all. A chain then runs in one pass (split only so that a pass's step
// count fits an int) and reconstruction tests for change every
// kSoloRecSteps steps.
// Fewest passes of a uint8 chain or program for the tagged hand-over: the
// planes are zeroed before the launch (about 2 us at 1024^2), which one
// hand-over does not repay (1024^2 opening of 2 passes: 25 us plain, 27 us
// tagged; 1500-step chain of 75 passes: 0.760 -> 0.725 ms).
constexpr int kTaggedMinPasses = 3;
constexpr int64_t kSoloPassSteps = (int64_t)1 << 30;
constexpr int kSoloRecSteps = 64;
__host__ __device__ inline int64_t rr_passes(int64_t steps, int K) {
  const int64_t k = K > 0 ? (int64_t)K : kSoloPassSteps;
  return (steps + k - 1) / k;
}

// Tile geometry of one launch: interior TH x TW, halo K, shared-memory row
// stride rs, tile grid, CTA count and dynamic shared memory.
struct Plan {
  int TH, TW, K, rs, tiles_x, tiles_y, grid;
  size_t smem;
  int variant;  // register kernel: shape variant (0 = default)
};
inline bool single_tile(const Plan &P, int batch) { return batch <= 1 && P.tiles_x == 1 && P.tiles_y == 1; }

// Tuned pass length K of the default kernel shape for an item-op code (0..5
// as geo_item.op), or 0 when the tune cache has no entry (geo_tune.cu). The
// entry of the exact (H, W) is used first, else that of its size class.
int tuned_k(int dt, int op, int conn, int64_t H, int64_t W, int64_t steps);
// The autotuner's planner override for the calling thread (geo_tune.cu sets
// it around each timed call, so tuning never touches the process
// environment): K > 0 forces the pass length, variant >= 0 the shape variant
// of the register kernel; {0, -1} = none (geo_api.cu).
struct PlanOverride {
  int K, variant;
};
PlanOverride &plan_override();
// Tuned (K, variant) over every kernel shape; false when there is no entry.
bool tuned_plan(int dt, int op, int conn, int64_t H, int64_t W, int64_t steps, int *K, int *variant);
// The batch planner's per-pass charge chosen by geo_batch_autotune (10 when
// untuned), and its setter (geo_tune.cu).
double tuned_batch_sync();
void set_tuned_batch_sync(double sync, float ms);

// Stream-ordered scratch from the library's per-device pool (geo_api.cu).
int pool_alloc(void **p, size_t n, cudaStream_t s);
int pool_free(void *p, cudaStream_t s);

// The per-device status word that device-side waits report into (geo_api.cu).
int device_status_word(int **status);
// Host-side failure injection read from GEOMORPH_FAULT (geo_api.cu).
enum HostFault { FAULT_NONE = 0, FAULT_BADARG, FAULT_ALLOC, FAULT_TIMEOUT };
HostFault host_fault();
// Read and clear the status word of the no-allocation chain on device `dev`
// (geo_noalloc.cu); 0 if that entry point has not run on the device. The
// caller has synchronised the stream. Allocates nothing.
int noalloc_take_status(int dev, int *status);

// Uncached tile planning and launch (geo_api.cu).
int plan_tiles(int dt, int op, int conn, int64_t H, int64_t W, int64_t steps_hint, int nsm, Plan *P, int batch = 1);

// Chain / reconstruction / window driver of the C ABI (geo_api.cu): a batch
// of equal-shape images stored one after another (image stride H * pitch).
int run_chain(int dt, const void *marker, const void *mask, void *out, int64_t H, int64_t W, int64_t pitch, int conn,
              int op, int mode, int64_t steps, int64_t *steps_out, void *stream, int batch);
int launch_plan(int dt, const TileLaunch &L, int op, int conn, cudaStream_t s, const Plan &P);
// The same driver for any element type including the internal GEO_D32 (no
// check of dt against the public geo_dtype values).
int run_chain_any(int dt, const void *marker, const void *mask, void *out, int64_t H, int64_t W, int64_t pitch,
                  int conn, int op, int mode, int64_t steps, int64_t *steps_out, void *stream, int batch);
// float64 through the rank transform (geo_rank.cu): whether it applies
// (size, chain length, GEOMORPH_F64=keys|ranks), and the driver.
bool rank_path_applies(int64_t H, int64_t W, bool has_mask, int mode, int64_t steps);
int run_chain_ranked(const double *marker, const double *mask, double *out, int64_t H, int64_t W, int64_t pitch,
                     int conn, int op, int mode, int64_t steps, int64_t *steps_out, void *stream);
// Cached plan of the register-resident kernel for an element type, op, item
// code (0..5 as geo_item.op, for the tune cache) and chain length hint.
int plan_rr(int dt, int op, int code, int conn, int64_t H, int64_t W, int64_t steps_hint, Plan *P);

// Host-side launcher per element type (defined in geo_tile_<dtype>.cu).

int launch_tile_u8(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid, size_t smem);
int launch_tile_f32(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid, size_t smem);
int launch_tile_f64(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid, size_t smem);
int launch_rr_u8(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid, int variant = 0);
int launch_rr_f32(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid, int variant = 0);
int launch_rr_f64(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid);
int occupancy_rr_u8(int op, int conn, int *blocks_per_sm, int variant = 0);
int occupancy_rr_f32(int op, int conn, int *blocks_per_sm, int variant = 0);
// the variant shapes, one translation unit each (geo_rr_u8_v<n>.cu, geo_rr_f32_v<n>.cu)
int launch_rr_u8_v1(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid);
int launch_rr_u8_v2(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid);
int occupancy_rr_u8_v1(int op, int conn, int *blocks_per_sm);
int occupancy_rr_u8_v2(int op, int conn, int *blocks_per_sm);
int launch_rr_f32_v1(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid);
int launch_rr_f32_v2(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid);
int occupancy_rr_f32_v1(int op, int conn, int *blocks_per_sm);
int occupancy_rr_f32_v2(int op, int conn, int *blocks_per_sm);
int occupancy_rr_f64(int op, int conn, int *blocks_per_sm);
int launch_rr_d32(const TileLaunch &L, int op, int conn, cudaStream_t s, int grid);
int occupancy_rr_d32(int op, int conn, int *blocks_per_sm);
int occupancy_tile_u8(int op, int conn, size_t smem, int *blocks_per_sm);
int occupancy_tile_f32(int op, int conn, size_t smem, int *blocks_per_sm);
int occupancy_tile_f64(int op, int conn, size_t smem, int *blocks_per_sm);

}  // namespace geo
