// geo_dilate_chain_noalloc: the geodesic dilation chain for callers that
// cannot allocate GPU memory.
//
// Some callers must not allocate device memory during a call: code that runs
// under a fixed memory budget owned by another allocator, real-time loops
// that must not reach the driver's allocator, or hosts whose device memory is
// fully reserved up front. geo_dilate_chain takes its ping-pong image and its
// control words from a stream-ordered pool, which can allocate. This entry
// point instead uses a fixed scratch array in device memory that the library
// defines statically, so a call allocates nothing: no cudaMalloc, no
// cudaMallocAsync, no pool, no host heap.
//
// Costs and limits:
//   - every GPU that loads the library holds kNoAllocScratchBytes of device
//     memory for this array until the process exits;
//   - the scratch image needs round_up(width * element_size, 16) * height
//     bytes; larger images are rejected with GEO_ERR_WORKSPACE;
//   - all calls share the one array: calls that overlap on the GPU (other
//     streams, other threads) race and corrupt each other's results, so the
//     caller must order them;
//   - the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress and plans the tiles; make that first call before
//     any stream capture;
//   - a device-side wait that expires (the kernel gives up instead of
//     hanging, and `out` is then incomplete) is recorded in a status word
//     inside the array; it stays set across calls until geo_device_status
//     reads and clears it, which needs no allocation either.
#include <climits>
#include <cstring>
#include <mutex>

#include "geo_common.cuh"

namespace geo {

// Largest scratch image this entry point accepts (16 MiB: a 4096 x 4096
// uint8 image, a 2048 x 2048 float32 image or a 1448 x 1448 float64 image).
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
// Header of the array: control words at [0, 128), cleared on every call;
// the sticky status word at kNoAllocStatusOffset, cleared only when read.
constexpr size_t kNoAllocHeaderBytes = 512;
constexpr size_t kNoAllocControlBytes = 128;
constexpr size_t kNoAllocStatusOffset = 128;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocHeaderBytes + kNoAllocScratchBytes];

namespace {

constexpr int kMaxDev = 64;
constexpr int kPlanSlots = 32;

struct NoAllocDevice {
  bool ready;
  char *base;  // device address of g_noalloc_scratch on this device
  int nsm;
};

struct PlanSlot {
  bool used;
  int dev, dt, conn;
  int64_t H, W, hint;
  Plan plan;
};

std::mutex g_na_mu;
NoAllocDevice g_na_dev[kMaxDev];
PlanSlot g_na_plans[kPlanSlots];
int g_na_next = 0;

bool is_aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

bool ranges_overlap(const void *a, const void *b, size_t n) {
  const char *x = (const char *)a, *y = (const char *)b;
  return x < y + n && y < x + n;
}

Plane plane(const void *p, int64_t pitch_b, int dt) {
  const size_t va = dt == GEO_U8 ? 8 : 16;
  Plane q;
  q.ptr = (char *)p;
  q.pitch_b = pitch_b;
  q.vec_ok = (p != nullptr && is_aligned(p, va) && pitch_b % (int64_t)va == 0) ? 1 : 0;
  return q;
}

// Once per device, with that device current: the device address of the
// static scratch array and the SM count.
int setup_device(int dev, NoAllocDevice **out) {
  NoAllocDevice &d = g_na_dev[dev];
  if (!d.ready) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) return GEO_ERR_CUDA;
    if (cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GEO_ERR_CUDA;
    d.base = (char *)ptr;
    d.ready = true;
  }
  *out = &d;
  return GEO_OK;
}

int cached_plan(int dev, int dt, int conn, int64_t H, int64_t W, int64_t steps, int nsm, Plan *P) {
  const int64_t hint = steps < 64 ? steps : 64;
  for (auto &s : g_na_plans) {
    if (s.used && s.dev == dev && s.dt == dt && s.conn == conn && s.H == H && s.W == W && s.hint == hint) {
      *P = s.plan;
      return GEO_OK;
    }
  }
  int rc = plan_tiles(dt, DILATE, conn, H, W, steps, nsm, P);
  if (rc != GEO_OK) return rc;
  PlanSlot &s = g_na_plans[g_na_next];
  g_na_next = (g_na_next + 1) % kPlanSlots;
  s = PlanSlot{true, dev, dt, conn, H, W, hint, *P};
  return GEO_OK;
}

}  // namespace

int noalloc_take_status(int dev, int *status) {
  *status = 0;
  char *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (dev >= 0 && dev < kMaxDev && g_na_dev[dev].ready) base = g_na_dev[dev].base;
  }
  if (!base) return GEO_OK;  // never ran on this device: nothing recorded
  int *word = (int *)(base + kNoAllocStatusOffset);
  if (cudaMemcpy(status, word, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GEO_ERR_CUDA;
  return cudaMemset(word, 0, sizeof(int)) == cudaSuccess ? GEO_OK : GEO_ERR_CUDA;
}

}  // namespace geo

using namespace geo;

extern "C" int geo_dilate_chain_noalloc(geo_dtype dtype, const void *marker, const void *mask, void *out,
                                        int64_t height, int64_t width, int64_t pitch, int conn, int64_t steps,
                                        void *stream) {
  const int dt = (int)dtype;
  const HostFault fault = host_fault();
  if (fault == FAULT_BADARG) return GEO_ERR_ARG;
  if (dt != GEO_U8 && dt != GEO_F32 && dt != GEO_F64) return GEO_ERR_DTYPE;
  if (height < 0 || width < 0 || pitch < width || (conn != 4 && conn != 8) || steps < 0) return GEO_ERR_ARG;
  if (height == 0 || width == 0) return GEO_OK;
  if (!marker || !mask || !out) return GEO_ERR_ARG;
  const int es = dt == GEO_U8 ? 1 : dt == GEO_F32 ? 4 : 8;
  if (!is_aligned(marker, es) || !is_aligned(mask, es) || !is_aligned(out, es)) return GEO_ERR_ALIGN;
  const int64_t pitch_b = pitch * es;
  const size_t span = (size_t)((height - 1) * pitch_b + width * es);
  if (ranges_overlap(mask, out, span)) return GEO_ERR_ARG;
  const bool alias = (marker == out);
  if (!alias && ranges_overlap(marker, out, span)) return GEO_ERR_ARG;
  const int64_t spitch_b = ((width * es + 15) / 16) * 16;
  if (spitch_b > (int64_t)kNoAllocScratchBytes || spitch_b * height > (int64_t)kNoAllocScratchBytes)
    return GEO_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (steps == 0) {
    if (alias) return GEO_OK;
    return cudaMemcpy2DAsync(out, pitch_b, marker, pitch_b, width * es, height, cudaMemcpyDeviceToDevice, s) ==
                   cudaSuccess
               ? GEO_OK
               : GEO_ERR_CUDA;
  }

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return GEO_ERR_CUDA;
  NoAllocDevice *d = nullptr;
  Plan P;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    int rc = setup_device(dev, &d);
    if (rc != GEO_OK) return rc;
    rc = cached_plan(dev, dt, conn, height, width, steps, d->nsm, &P);
    if (rc != GEO_OK) return rc;
  }

  int64_t np = (steps + P.K - 1) / P.K;
  if (alias && (np & 1)) ++np;  // pass 0 must not write the buffer it reads
  if (np > INT_MAX) return GEO_ERR_ARG;  // TileLaunch::npasses is an int

  // layout of the static array: [0, 128) control words, cleared on every
  // call; the status word at offset 128, sticky until geo_device_status
  // reads it; [512, ...) the scratch image
  char *ctl = d->base;
  if (cudaMemsetAsync(ctl, 0, kNoAllocControlBytes, s) != cudaSuccess) return GEO_ERR_CUDA;

  TileLaunch L;
  memset(&L, 0, sizeof(L));
  L.marker = plane(marker, pitch_b, dt);
  L.mask = plane(mask, pitch_b, dt);
  L.out = plane(out, pitch_b, dt);
  L.scratch = plane(d->base + kNoAllocHeaderBytes, spitch_b, dt);
  L.H = height;
  L.W = width;
  L.TH = P.TH;
  L.TW = P.TW;
  L.K = P.K;
  L.tiles_x = P.tiles_x;
  L.tiles_y = P.tiles_y;
  L.rs = P.rs;
  L.mode = MODE_CHAIN;
  L.steps = steps;
  // GEOMORPH_FAULT=timeout: every wait on another CTA waits for something
  // that never happens and expires after a short limit (host-side injection)
  L.fault = fault == FAULT_TIMEOUT ? 1 : 0;
  L.wait_ns = L.fault ? kFaultWaitNs : kWaitLimitNs;
  L.npasses = (int)np;
  L.ctl = (Control *)ctl;
  L.status = (int *)(d->base + kNoAllocStatusOffset);
  L.steps_out = nullptr;
  return launch_plan(dt, L, DILATE, conn, s, P);
}
