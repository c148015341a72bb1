// extern "C" entry points of libgeomorph.so: argument checks, tile planning,
// scratch management, launch. Declarations and contracts: include/geomorph.h.
#include <cstdio>
#include <cstdlib>
#include <climits>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "geo_common.cuh"

namespace geo {

// ---------------------------------------------------------------------------
// per-device state: status word and a scratch memory pool
// ---------------------------------------------------------------------------

constexpr int kMaxDevices = 64;

struct DeviceState {
  bool init = false;
  int *status = nullptr;        // sticky device-side error word
  int *status_host = nullptr;   // pinned host slot the word is read into
  cudaMemPool_t pool = nullptr;  // library-owned stream-ordered pool
  int nsm = 0;
};

static std::mutex g_mu;
static DeviceState g_dev[kMaxDevices];

static int device_state(DeviceState **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GEO_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceState &d = g_dev[dev];
  if (!d.init) {
    if (cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GEO_ERR_CUDA;
    if (cudaMalloc(&d.status, sizeof(int)) != cudaSuccess) return GEO_ERR_CUDA;
    if (cudaMemset(d.status, 0, sizeof(int)) != cudaSuccess) return GEO_ERR_CUDA;
    if (cudaMallocHost(&d.status_host, sizeof(int)) != cudaSuccess) return GEO_ERR_CUDA;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&d.pool, &props) != cudaSuccess) return GEO_ERR_CUDA;
    uint64_t thr = UINT64_MAX;  // keep freed scratch cached in the pool
    cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &thr);
    d.init = true;
  }
  *out = &d;
  return GEO_OK;
}

int pool_alloc(void **p, size_t n, cudaStream_t s) {
  DeviceState *ds = nullptr;
  const int rc = device_state(&ds);
  if (rc != GEO_OK) return rc;
  return cudaMallocFromPoolAsync(p, n, ds->pool, s) == cudaSuccess ? GEO_OK : GEO_ERR_CUDA;
}

int pool_free(void *p, cudaStream_t s) { return cudaFreeAsync(p, s) == cudaSuccess ? GEO_OK : GEO_ERR_CUDA; }

int device_status_word(int **status) {
  DeviceState *ds = nullptr;
  const int rc = device_state(&ds);
  if (rc != GEO_OK) return rc;
  *status = ds->status;
  return GEO_OK;
}

// ---------------------------------------------------------------------------
// planning
// ---------------------------------------------------------------------------

static int elem_size(int dt) { return dt == GEO_U8 ? 1 : (dt == GEO_F32 || dt == GEO_D32) ? 4 : 8; }
static int chunk_elems(int dt) { return dt == GEO_U8 ? 8 : dt == GEO_F32 ? 4 : 2; }

static int occupancy(int dt, int op, int conn, size_t smem, int *bps) {
  if (dt == GEO_U8) return occupancy_tile_u8(op, conn, smem, bps);
  if (dt == GEO_F32) return occupancy_tile_f32(op, conn, smem, bps);
  return occupancy_tile_f64(op, conn, smem, bps);
}

static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Choose the tile interior TH x TW and halo K. The cost model per step is
// (waves of tiles) x (area a tile computes per step, about (TH+K)(TW+K)),
// plus a fixed synchronisation cost per pass spread over the pass's K steps.
int plan_tiles(int dt, int op, int conn, int64_t H, int64_t W, int64_t steps_hint, int nsm, Plan *P, int batch) {
  const int CE = chunk_elems(dt);
  int Kmax = dt == GEO_U8 ? 24 : dt == GEO_F32 ? 12 : 6;
  if (const char *e = getenv("GEOMORPH_K")) Kmax = atoi(e);
  int K = Kmax;
  if (steps_hint > 0 && steps_hint < K) K = (int)steps_hint;
  K = ((K + CE - 1) / CE) * CE;
  if (K < CE) K = CE;
  const int SS = dt == GEO_U8 ? 2 : elem_size(dt);
  const double sync_px = 6000.0;  // barrier cost per pass, in pixel-steps of one SM
  double best = 1e300;
  Plan bp{};
  static const int cand_th[] = {16, 24, 32, 40, 48, 56, 64, 72, 80, 88, 96, 112, 128, 160, 192, 256};
  static const int cand_tw[] = {16, 24, 32, 40, 48, 56, 64, 72, 80, 88, 96, 112, 128, 160, 192, 256};
  for (int th : cand_th) {
    for (int tw : cand_tw) {
      if (tw % CE) continue;
      const int RH = th + 2 * K;
      const int NC = (tw + 2 * K) / CE + 2;
      int rs = NC * 16;
      if (rs % 128 == 0) rs += 16;
      const size_t smem = (size_t)3 * RH * rs;
      if (smem > 200 * 1024) continue;
      int bps = 0;
      if (occupancy(dt, op, conn, smem, &bps) != GEO_OK) return GEO_ERR_CUDA;
      if (bps <= 0) continue;
      const int64_t tiles = cdiv(H, th) * cdiv(W, tw) * batch;
      const int64_t slots = (int64_t)bps * nsm;
      const int64_t grid = tiles < slots ? tiles : slots;
      // tiles share an SM when more than one CTA is resident per SM
      const double per_sm = (double)cdiv(tiles, nsm);
      const double area = (double)(th + K) * (double)(tw + K) * SS;
      const double cost = per_sm * area + sync_px * SS / K;
      if (cost < best) {
        best = cost;
        bp.TH = th;
        bp.TW = tw;
        bp.K = K;
        bp.rs = rs;
        bp.tiles_x = (int)cdiv(W, tw);
        bp.tiles_y = (int)cdiv(H, th);
        bp.grid = (int)grid;
        bp.smem = smem;
      }
    }
  }
  if (best >= 1e300) return GEO_ERR_CUDA;
  if (const char *e = getenv("GEOMORPH_TILE")) {  // "THxTW" override for tuning sweeps
    int th = 0, tw = 0;
    if (sscanf(e, "%dx%d", &th, &tw) == 2 && th > 0 && tw > 0 && tw % CE == 0) {
      const int RH = th + 2 * K;
      const int NC = (tw + 2 * K) / CE + 2;
      int rs = NC * 16;
      if (rs % 128 == 0) rs += 16;
      const size_t smem = (size_t)3 * RH * rs;
      int bps = 0;
      if (smem <= 227 * 1024 && occupancy(dt, op, conn, smem, &bps) == GEO_OK && bps > 0) {
        const int64_t tiles = cdiv(H, th) * cdiv(W, tw) * batch;
        const int64_t slots = (int64_t)bps * nsm;
        bp = Plan{th, tw, K, rs, (int)cdiv(W, tw), (int)cdiv(H, th), (int)(tiles < slots ? tiles : slots), smem};
      }
    }
  }
  *P = bp;
  return GEO_OK;
}

using PlanKey = std::tuple<int, int, int, int, int64_t, int64_t, int64_t, int, std::string, std::string>;
static std::map<PlanKey, Plan> g_plans;
static std::mutex g_plan_mu;

static int make_plan(int dt, int op, int conn, int64_t H, int64_t W, int64_t steps_hint, int nsm, Plan *P,
                     int batch) {
  int dev = 0;
  cudaGetDevice(&dev);
  const char *ek = getenv("GEOMORPH_K");
  const char *et = getenv("GEOMORPH_TILE");
  PlanKey key{dev * 1024 + batch, dt, op, conn, H, W, steps_hint < 64 ? steps_hint : 64, nsm, ek ? ek : "", et ? et : ""};
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) {
      *P = it->second;
      return GEO_OK;
    }
  }
  int rc = plan_tiles(dt, op, conn, H, W, steps_hint, nsm, P, batch);
  if (rc == GEO_OK && getenv("GEOMORPH_DEBUG"))
    fprintf(stderr, "geomorph plan: dt=%d op=%d conn=%d %lldx%lld -> tile %dx%d K=%d tiles=%dx%d grid=%d smem=%zu\n",
            dt, op, conn, (long long)H, (long long)W, P->TH, P->TW, P->K, P->tiles_y, P->tiles_x, P->grid, P->smem);
  if (rc == GEO_OK) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans[key] = *P;
  }
  return rc;
}

// ---------------------------------------------------------------------------
// register-resident kernel: fixed region per element type, K chosen here
// ---------------------------------------------------------------------------

struct RRGeom {
  int CW, RW, NW, B;
};
// must match SU8 / SF32 / SF64 and their variants in geo_rr.cuh (CW, RW, NW, bands)
static RRGeom rr_geom(int dt, int variant = 0) {
  if (dt == GEO_U8 && variant == 1) return RRGeom{4, GEO_RR_U8_V1_RW, GEO_RR_U8_V1_NW, 2};
  if (dt == GEO_U8 && variant == 2) return RRGeom{4, GEO_RR_U8_V2_RW, GEO_RR_U8_V2_NW, 2};
  if (dt == GEO_U8 || dt == GEO_D32) return RRGeom{4, GEO_RR_U8_RW, GEO_RR_U8_NW, 2};
  if (dt == GEO_F32 && variant == 1) return RRGeom{4, GEO_RR_F32_V1_RW, GEO_RR_F32_V1_NW, 1};
  if (dt == GEO_F32 && variant == 2) return RRGeom{4, GEO_RR_F32_V2_RW, GEO_RR_F32_V2_NW, 1};
  if (dt == GEO_F32) return RRGeom{4, GEO_RR_F32_RW, GEO_RR_F32_NW, 1};
  return RRGeom{2, GEO_RR_F64_RW, GEO_RR_F64_NW, 1};
}

// shape variants an element type has (uint8 and float32: kRRVariants)
static int rr_variants(int dt) { return (dt == GEO_U8 || dt == GEO_F32) ? kRRVariants : 1; }

static int occupancy_rr(int dt, int op, int conn, int *bps, int variant = 0) {
  if (dt == GEO_U8) return occupancy_rr_u8(op, conn, bps, variant);
  if (dt == GEO_D32) return occupancy_rr_d32(op, conn, bps);
  if (dt == GEO_F32) return occupancy_rr_f32(op, conn, bps, variant);
  return occupancy_rr_f64(op, conn, bps);
}

// Pick the halo K of the register-resident kernel. Cost model in units of
// one region-step (one step of one CTA on its whole region): a pass costs
// kSyncSteps for its load / store / grid barrier, and every step costs one
// unit per tile an SM has to process in that pass.
PlanOverride &plan_override() {
  thread_local PlanOverride o{0, -1};
  return o;
}

// forceK > 0: that pass length (an override or the tune table), else the
// cost model's choice
static int plan_rr_uncached(int dt, int op, int conn, int64_t H, int64_t W, int64_t steps_hint, int nsm, Plan *P,
                            int batch, int forceK, int variant) {
  const RRGeom g = rr_geom(dt, variant);
  const int RWID = 32 * g.CW, RHGT = g.NW * g.RW * g.B;
  int bps = 0;
  if (occupancy_rr(dt, op, conn, &bps, variant) != GEO_OK || bps <= 0) return GEO_ERR_CUDA;
  double kSyncSteps = 10.0;
  if (const char *e = getenv("GEOMORPH_SYNC")) kSyncSteps = atof(e);
  double best = 1e300;
  Plan bp{};
  // K <= min(TH, TW): a tile's halo then reaches only its 8 neighbours,
  // which is what the point-to-point pass synchronisation assumes
  const int kmax = (RWID < RHGT ? RWID : RHGT) / 3;
  for (int K = g.CW; K <= kmax; K += g.CW) {
    if (forceK > 0 && K != ((forceK + g.CW - 1) / g.CW) * g.CW) continue;
    const int TW = RWID - 2 * K, TH = RHGT - 2 * K;
    const int64_t tiles = cdiv(H, TH) * cdiv(W, TW) * batch;
    // blocks resident at once: a step of one region takes one unit of an SM
    // per resident block (bps > 1 only for the small variants)
    const double per_sm = (double)cdiv(tiles, (int64_t)nsm * bps) * bps;
    // one tile covering one image runs without pass boundaries (rr_passes)
    const bool one = tiles == 1;
    double cost;
    if (steps_hint > 0) {
      const double passes = one ? 1.0 : (double)cdiv(steps_hint, K);
      cost = passes * kSyncSteps * per_sm + per_sm * (double)steps_hint;
    } else if (one) {
      const double n = (double)(H > W ? H : W);
      cost = n + kSoloRecSteps + (n / kSoloRecSteps + 2.0) * kSyncSteps;
    } else {
      // reconstruction: the step count is unknown; take the longest side as
      // its scale and charge the overshoot (the pass that ends past the fixed
      // point and the pass that detects it, about 1.5 K steps)
      const double n = (double)(H > W ? H : W);
      cost = per_sm * (n + 1.5 * K) + (n / K + 2.0) * kSyncSteps * per_sm;
    }
    if (cost < best) {
      best = cost;
      const int64_t slots = (int64_t)bps * nsm;
      bp = Plan{TH, TW, K, 0, (int)cdiv(W, TW), (int)cdiv(H, TH), (int)(tiles < slots ? tiles : slots), 0, variant};
      (void)batch;
    }
  }
  if (best >= 1e300) return GEO_ERR_ARG;
  *P = bp;
  return GEO_OK;
}

using RRPlanKey = std::tuple<int, int, int, int, int, int64_t, int64_t, int64_t, int, std::string, int, int>;
static std::map<RRPlanKey, Plan> g_rr_plans;

// code: the operation as a geo_item.op code (0..5), for the tune cache.
// variants: whether the plan may use a shape variant of the kernel (the
// chains, reconstructions and windows of run_chain_any); the other kernels
// built on the same region (programs, the distance transform) take the
// default shape and the tuned K of that shape.
static int make_plan_rr(int dt, int op, int code, int conn, int64_t H, int64_t W, int64_t steps_hint, int nsm,
                        Plan *P, int batch, bool variants = false) {
  int dev = 0;
  cudaGetDevice(&dev);
  const char *es = getenv("GEOMORPH_SYNC");
  // the pass length and shape: the autotuner's per-thread override, else the
  // GEOMORPH_K / GEOMORPH_VARIANT environment overrides (sweeps), else the
  // tune table, else the cost model (K = 0) in the default shape
  const PlanOverride &ov = plan_override();
  const char *ek = getenv("GEOMORPH_K");
  const char *ev = getenv("GEOMORPH_VARIANT");
  const int oK = ov.K > 0 ? ov.K : (ek ? atoi(ek) : 0);
  const int oV = ov.variant >= 0 ? ov.variant : (ev ? atoi(ev) : -1);
  int tk = 0, tv = 0;
  if (variants && oV >= 0) {
    tk = oK;
    tv = oV;
    if (tv >= rr_variants(dt)) return GEO_ERR_ARG;
  } else if (oK > 0) {
    tk = oK;
  } else if (variants && batch == 1) {
    if (!tuned_plan(dt, code, conn, H, W, steps_hint, &tk, &tv) || tv < 0 || tv >= rr_variants(dt)) tk = tv = 0;
  } else {
    tk = tuned_k(dt, code, conn, H, W, steps_hint);
  }
  RRPlanKey key{dev, batch, dt, op, conn, H, W, steps_hint, nsm, es ? es : "", tk, tv};
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_rr_plans.find(key);
    if (it != g_rr_plans.end()) {
      *P = it->second;
      return GEO_OK;
    }
  }
  int rc = plan_rr_uncached(dt, op, conn, H, W, steps_hint, nsm, P, batch, tk, tv);
  if (rc == GEO_OK && getenv("GEOMORPH_DEBUG"))
    fprintf(stderr, "geomorph rr plan: dt=%d op=%d conn=%d %lldx%lld steps=%lld -> interior %dx%d K=%d tiles=%dx%d grid=%d variant=%d\n",
            dt, op, conn, (long long)H, (long long)W, (long long)steps_hint, P->TH, P->TW, P->K, P->tiles_y,
            P->tiles_x, P->grid, P->variant);
  if (rc == GEO_OK) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_rr_plans[key] = *P;
  }
  return rc;
}

static int launch_rr(int dt, const TileLaunch &L, int op, int conn, cudaStream_t s, const Plan &P) {
  if (dt == GEO_U8) return launch_rr_u8(L, op, conn, s, P.grid, P.variant);
  if (dt == GEO_D32) return launch_rr_d32(L, op, conn, s, P.grid);
  if (dt == GEO_F32) return launch_rr_f32(L, op, conn, s, P.grid, P.variant);
  return launch_rr_f64(L, op, conn, s, P.grid);
}

int launch_plan(int dt, const TileLaunch &L, int op, int conn, cudaStream_t s, const Plan &P) {
  if (dt == GEO_U8) return launch_tile_u8(L, op, conn, s, P.grid, P.smem);
  if (dt == GEO_F32) return launch_tile_f32(L, op, conn, s, P.grid, P.smem);
  return launch_tile_f64(L, op, conn, s, P.grid, P.smem);
}

static bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

static Plane make_plane(const void *p, int64_t pitch_b, int dt, bool rr) {
  // width of the kernel's vector access: 16-byte chunks (8 bytes for u8) in
  // the shared-memory kernel, CW pixels per lane in the register kernel
  const size_t va = rr ? (size_t)rr_geom(dt).CW * elem_size(dt) : (dt == GEO_U8 ? 8 : 16);
  Plane q;
  q.ptr = (char *)p;
  q.pitch_b = pitch_b;
  q.vec_ok = (p != nullptr && aligned(p, va) && pitch_b % (int64_t)va == 0) ? 1 : 0;
  return q;
}

static bool overlaps(const void *a, const void *b, size_t n) {
  const char *x = (const char *)a, *y = (const char *)b;
  return x < y + n && y < x + n;
}

int plan_rr(int dt, int op, int code, int conn, int64_t H, int64_t W, int64_t steps_hint, Plan *P) {
  DeviceState *ds = nullptr;
  const int rc = device_state(&ds);
  if (rc != GEO_OK) return rc;
  return make_plan_rr(dt, op, code, conn, H, W, steps_hint, ds->nsm, P, 1);
}

// Common driver of chains, reconstruction and windows (public element types).
int run_chain(int dt, const void *marker, const void *mask, void *out, int64_t H, int64_t W, int64_t pitch, int conn,
              int op, int mode, int64_t steps, int64_t *steps_out, void *stream, int batch) {
  if (dt != GEO_U8 && dt != GEO_F32 && dt != GEO_F64) return GEO_ERR_DTYPE;
  return run_chain_any(dt, marker, mask, out, H, W, pitch, conn, op, mode, steps, steps_out, stream, batch);
}

// Failure injection on the host (GEOMORPH_FAULT), for testing how failures
// are reported without faulting a GPU: "badarg" rejects the call as an
// invalid argument, "alloc" fails the scratch allocation, and "timeout"
// launches normally but makes every wait on another CTA (neighbour epochs,
// grid barrier) wait for something that never happens, so that it expires
// after kFaultWaitNs and the kernel records GEO_ERR_TIMEOUT and returns.
HostFault host_fault() {
  const char *e = getenv("GEOMORPH_FAULT");
  if (!e) return FAULT_NONE;
  if (strcmp(e, "badarg") == 0) return FAULT_BADARG;
  if (strcmp(e, "alloc") == 0) return FAULT_ALLOC;
  if (strcmp(e, "timeout") == 0) return FAULT_TIMEOUT;
  return FAULT_NONE;
}

int run_chain_any(int dt, const void *marker, const void *mask, void *out, int64_t H, int64_t W, int64_t pitch,
                  int conn, int op, int mode, int64_t steps, int64_t *steps_out, void *stream, int batch) {
  // rank codes run as float32 (same kernels and planes) and may take the
  // tagged hand-over in the default shape
  const bool rank_codes = (dt == GEO_R32);
  if (rank_codes) dt = GEO_F32;
  const HostFault fault = host_fault();
  if (fault == FAULT_BADARG) return GEO_ERR_ARG;
  if (batch < 1) return GEO_ERR_ARG;
  if (H < 0 || W < 0 || pitch < W || (conn != 4 && conn != 8) || (op != DILATE && op != ERODE))
    return GEO_ERR_ARG;
  if (H == 0 || W == 0) return GEO_OK;
  if (!marker || !out) return GEO_ERR_ARG;
  const int es = elem_size(dt);
  if (!aligned(marker, es) || !aligned(out, es) || (mask && !aligned(mask, es))) return GEO_ERR_ALIGN;
  const int64_t pitch_b = pitch * es;
  const size_t span = (size_t)((int64_t)(batch - 1) * H * pitch_b + (H - 1) * pitch_b + W * es);
  if (mask && overlaps(mask, out, span)) return GEO_ERR_ARG;
  const bool alias = (marker == out);
  if (!alias && overlaps(marker, out, span)) return GEO_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;

  if (mode == MODE_CHAIN && steps == 0) {
    if (alias) return GEO_OK;
    return cudaMemcpy2DAsync(out, pitch_b, marker, pitch_b, W * es, H * (int64_t)batch, cudaMemcpyDeviceToDevice,
                             s) == cudaSuccess
               ? GEO_OK
               : GEO_ERR_CUDA;
  }

  // float64: long chains and reconstructions run on the ranks of the values
  // (an injected allocation failure is tested on the direct path; an
  // injected timeout reaches the rank path's chain)
  if (dt == GEO_F64 && batch == 1 && (fault == FAULT_NONE || fault == FAULT_TIMEOUT) &&
      rank_path_applies(H, W, mask != nullptr, mode, steps))
    return run_chain_ranked((const double *)marker, (const double *)mask, (double *)out, H, W, pitch, conn, op, mode,
                            steps, steps_out, stream);

  DeviceState *ds = nullptr;
  int rc = device_state(&ds);
  if (rc != GEO_OK) return rc;
  const char *kern = getenv("GEOMORPH_KERNEL");
  const bool rr = !(kern && strcmp(kern, "tile") == 0) || dt == GEO_D32;  // the distances have no tile kernel
  Plan P;
  const int code = mode == MODE_REC ? 2 + op : (mask ? op : 4 + op);
  rc = rr ? make_plan_rr(dt, op, code, conn, H, W, mode == MODE_CHAIN ? steps : 0, ds->nsm, &P, batch, !rank_codes)
          : make_plan(dt, op, conn, H, W, mode == MODE_CHAIN ? steps : 0, ds->nsm, &P, batch);
  if (rc != GEO_OK) return rc;

  // scratch: control words (+ per-tile pass epochs of the register kernel)
  // and one ping-pong image with a 16-byte aligned pitch
  const int64_t spitch_b = ((W * es + 15) / 16) * 16;
  const size_t ntiles = (size_t)P.tiles_x * (size_t)P.tiles_y * (size_t)batch;
  // [control 256 B][per-tile pass epochs][per-tile changed flags, two passes]
  // [tagged reconstruction: pass ring of votes and outcomes; abort flag]
  const size_t ring_b = ((2 * (size_t)kRecRing + 1) * sizeof(int) + 255) / 256 * 256;
  const size_t ctl_b = 256 + ((3 * ntiles * sizeof(int) + 255) / 256) * 256 + (mode == MODE_REC ? ring_b : 0);
  int64_t np = 0;
  if (mode == MODE_CHAIN) {
    np = rr ? rr_passes(steps, single_tile(P, batch) ? 0 : P.K) : cdiv(steps, P.K);
    if (alias && (np & 1)) ++np;  // pass 0 must not write the buffer it reads
    if (np > INT_MAX) return GEO_ERR_ARG;  // TileLaunch::npasses is an int
  }
  // uint8 and rank-code chains of several passes with one tile per CTA hand
  // the passes over in two zeroed planes of tagged words (GEOMORPH_TAGGED=0:
  // plain planes and tile epochs); the lane's 4 columns must be whole words.
  // From 3 passes on: zeroing the planes costs about as much as one
  // hand-over saves. Reconstruction of several tiles, one per CTA, hands
  // over the same way and finds its fixed point without a grid barrier
  // (rr_kernel). uint8 words: 8 bytes per 4 pixels; rank-code words: 4 bytes
  // per pixel, rows padded to 4 words (16-byte accesses).
  const char *tg = getenv("GEOMORPH_TAGGED");
  const bool tagged = rr && (dt == GEO_U8 || (rank_codes && P.variant == 0)) && batch == 1 &&
                      ((mode == MODE_CHAIN && np >= kTaggedMinPasses) || (mode == MODE_REC && ntiles >= 2)) &&
                      ntiles <= (size_t)P.grid && P.K % 4 == 0 && P.TW % 4 == 0 && !(tg && strcmp(tg, "0") == 0);
  const int64_t tpitch = rank_codes ? (W + 3) / 4 * 4 : (W + 3) / 4;
  const size_t tword_b = rank_codes ? 4 : 8;
  const size_t tag_b = tagged ? ((2 * (size_t)tpitch * (size_t)H * tword_b + 255) / 256) * 256 : 0;
  const size_t scratch_b = ctl_b + tag_b + (size_t)spitch_b * (size_t)H * (size_t)batch;
  // A register-kernel chain of one pass (a single-tile image, or a short
  // chain) reads the marker and writes out once: no ping-pong image, no
  // pass epochs, no control words, so no scratch and no memset.
  const bool one_pass = rr && mode == MODE_CHAIN && np == 1;
  void *scratch = nullptr;
  if (fault == FAULT_ALLOC) return GEO_ERR_CUDA;
  if (!one_pass && cudaMallocFromPoolAsync(&scratch, scratch_b, ds->pool, s) != cudaSuccess) return GEO_ERR_CUDA;
  rc = GEO_OK;
  if (!one_pass && cudaMemsetAsync(scratch, 0, ctl_b + tag_b, s) != cudaSuccess) rc = GEO_ERR_CUDA;

  TileLaunch L;
  memset(&L, 0, sizeof(L));
  L.marker = make_plane(marker, pitch_b, dt, rr);
  L.mask = make_plane(mask, pitch_b, dt, rr);
  L.out = make_plane(out, pitch_b, dt, rr);
  L.scratch = make_plane(one_pass ? nullptr : (char *)scratch + ctl_b + tag_b, spitch_b, dt, rr);
  L.marker.bstride = L.out.bstride = H * pitch_b;
  L.mask.bstride = mask ? H * pitch_b : 0;
  L.scratch.bstride = H * spitch_b;
  L.batch = batch;
  L.H = H;
  L.W = W;
  L.TH = P.TH;
  L.TW = P.TW;
  L.K = P.K;
  L.tiles_x = P.tiles_x;
  L.tiles_y = P.tiles_y;
  L.rs = P.rs;
  L.mode = mode;
  L.steps = steps;
  L.alias = alias ? 1 : 0;
  L.ctl = (Control *)scratch;
  L.epoch = one_pass ? nullptr : (int *)((char *)scratch + 256);
  L.tchg = one_pass ? nullptr : L.epoch + ntiles;
  L.status = ds->status;
  L.steps_out = steps_out;
  L.fault = fault == FAULT_TIMEOUT ? 1 : 0;
  L.wait_ns = L.fault ? kFaultWaitNs : kWaitLimitNs;
  if (mode == MODE_CHAIN) L.npasses = (int)np;
  if (tagged) {
    L.tagged = (unsigned long long *)((char *)scratch + ctl_b);
    L.tpitch = tpitch;
    L.tplane = tpitch * H;
  }
  if (mode == MODE_REC) {
    char *ring = (char *)scratch + ctl_b - ring_b;
    L.rec_done = (int *)ring;
    L.rec_res = (unsigned *)(L.rec_done + kRecRing);
    L.rec_abort = (int *)(L.rec_res + kRecRing);
  }
  if (rc == GEO_OK) rc = rr ? launch_rr(dt, L, op, conn, s, P) : launch_plan(dt, L, op, conn, s, P);
  if (scratch && cudaFreeAsync(scratch, s) != cudaSuccess && rc == GEO_OK) rc = GEO_ERR_CUDA;
  return rc;
}

}  // namespace geo

using namespace geo;

extern "C" {

const char *geo_status_string(int status) {
  switch (status) {
    case GEO_OK: return "GEO_OK";
    case GEO_ERR_ARG: return "GEO_ERR_ARG: invalid argument";
    case GEO_ERR_DTYPE: return "GEO_ERR_DTYPE: unsupported element type";
    case GEO_ERR_ALIGN: return "GEO_ERR_ALIGN: misaligned pointer";
    case GEO_ERR_CUDA: return "GEO_ERR_CUDA: CUDA runtime error";
    case GEO_ERR_TIMEOUT: return "GEO_ERR_TIMEOUT: device wait expired";
    case GEO_ERR_NOT_CONVERGED: return "GEO_ERR_NOT_CONVERGED: reconstruction hit max_steps";
    case GEO_ERR_WORKSPACE: return "GEO_ERR_WORKSPACE: workspace too small";
    default: return "unknown geo_status";
  }
}

int geo_plan_info(geo_dtype dtype, int op, int conn, int64_t height, int64_t width, int64_t steps, int *K, int *TH,
                  int *TW) {
  return geo_plan_shape(dtype, op, conn, height, width, steps, K, TH, TW, nullptr, nullptr);
}

int geo_plan_shape(geo_dtype dtype, int op, int conn, int64_t height, int64_t width, int64_t steps, int *K, int *TH,
                   int *TW, int *variant, int *threads) {
  if (dtype != GEO_U8 && dtype != GEO_F32 && dtype != GEO_F64) return GEO_ERR_DTYPE;
  if (op < 0 || op > 5 || height <= 0 || width <= 0 || (op < 4 && conn != 4 && conn != 8)) return GEO_ERR_ARG;
  DeviceState *ds = nullptr;
  int rc = device_state(&ds);
  if (rc != GEO_OK) return rc;
  const bool rec = (op == 2 || op == 3);
  const int eop = (op == 1 || op == 3 || op == 5) ? ERODE : DILATE;
  Plan P;
  rc = make_plan_rr(dtype, eop, op, op >= 4 ? 8 : conn, height, width, rec ? 0 : steps, ds->nsm, &P, 1, true);
  if (rc != GEO_OK) return rc;
  if (K) *K = P.K;
  if (TH) *TH = P.TH;
  if (TW) *TW = P.TW;
  if (variant) *variant = P.variant;
  if (threads) *threads = rr_geom(dtype, P.variant).NW * 32;
  return GEO_OK;
}

int geo_device_status(void *stream, int *status) {
  if (!status) return GEO_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GEO_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  // the library's word, if this device has one (no device state is created
  // here, so a caller of the no-allocation chain allocates nothing by asking)
  int *word = nullptr, *host = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_dev[dev].init) {
      word = g_dev[dev].status;
      host = g_dev[dev].status_host;
    }
  }
  // read and clear in the stream's order after its work, one synchronisation
  // (the pinned slot is shared by the device's readers: one at a time)
  static std::mutex read_mu;
  std::lock_guard<std::mutex> rl(read_mu);
  if (word) {
    if (cudaMemcpyAsync(host, word, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GEO_ERR_CUDA;
    if (cudaMemsetAsync(word, 0, sizeof(int), s) != cudaSuccess) return GEO_ERR_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return GEO_ERR_CUDA;
  const int v = word ? *host : 0;
  // and the no-allocation chain's word
  int w = 0;
  if (noalloc_take_status(dev, &w) != GEO_OK) return GEO_ERR_CUDA;
  *status = v != 0 ? v : w;
  return GEO_OK;
}

int geo_dilate_chain(geo_dtype dtype, const void *marker, const void *mask, void *out, int64_t height,
                     int64_t width, int64_t pitch, int conn, int64_t steps, void *stream) {
  if (steps < 0 || (!mask && height > 0 && width > 0)) return GEO_ERR_ARG;
  return run_chain(dtype, marker, mask, out, height, width, pitch, conn, DILATE, MODE_CHAIN, steps, nullptr, stream, 1);
}

int geo_erode_chain(geo_dtype dtype, const void *marker, const void *mask, void *out, int64_t height,
                    int64_t width, int64_t pitch, int conn, int64_t steps, void *stream) {
  if (steps < 0 || (!mask && height > 0 && width > 0)) return GEO_ERR_ARG;
  return run_chain(dtype, marker, mask, out, height, width, pitch, conn, ERODE, MODE_CHAIN, steps, nullptr, stream, 1);
}

int geo_reconstruct(geo_dtype dtype, const void *marker, const void *mask, void *out, int64_t height,
                    int64_t width, int64_t pitch, int conn, int op, int64_t max_steps, int64_t *steps_out,
                    void *stream) {
  if (op != 0 && op != 1) return GEO_ERR_ARG;
  if (!mask && height > 0 && width > 0) return GEO_ERR_ARG;
  // default cap: every changing step of any input (at most H*W + 1) plus room
  // for the last, unchanged pass that detects the fixed point (K <= 1024)
  if (max_steps <= 0) max_steps = height * width + 1 + 1024;
  return run_chain(dtype, marker, mask, out, height, width, pitch, conn, op, MODE_REC, max_steps, steps_out, stream,
                   1);
}

int morph_window_dilate(geo_dtype dtype, const void *in, void *out, int64_t height, int64_t width, int64_t pitch,
                        int64_t half_size, void *stream) {
  if (half_size < 0) return GEO_ERR_ARG;
  return run_chain(dtype, in, nullptr, out, height, width, pitch, 8, DILATE, MODE_CHAIN, half_size, nullptr, stream, 1);
}

int morph_window_erode(geo_dtype dtype, const void *in, void *out, int64_t height, int64_t width, int64_t pitch,
                       int64_t half_size, void *stream) {
  if (half_size < 0) return GEO_ERR_ARG;
  return run_chain(dtype, in, nullptr, out, height, width, pitch, 8, ERODE, MODE_CHAIN, half_size, nullptr, stream, 1);
}

}  // extern "C"
