// Measured choice of the register kernel's shape and pass length per
// (element type, operation, connectivity, image size, chain length class),
// persisted in a small text file.
//
// What is tuned: the pass length K (the halo, which fixes the tile interior)
// and the shape variant of the register-resident kernel (band height, warps
// per block, hence region and block size; geo_common.cuh). Each entry keeps
// the fastest (K, variant) over every variant and, separately, the fastest K
// of the default shape (K0), which the kernels that exist in the default
// shape only use (the batch kernel, programs, the distance transform).
//
// Keys. An entry is made for the exact (height, width) tuned and one for its
// size class: height and width in half-octave classes, floor(2 log2 n). The
// planners look for the exact entry first, then the class entry, and fall
// back to their cost model; the class entry of a class comes from the
// largest item tuned in it. steps_class is the chain length when it is below
// 64 (there K may exceed the length) and 64 otherwise; reconstructions use -1.
//
// File (version 2): a header "geomorph-tune 2 <device name>", then lines
//   E dtype op conn height width steps_class K variant ms K0 ms0
//   C dtype op conn hclass wclass steps_class K variant ms K0 ms0 work
//   B sync ms            (the batch planner's per-pass charge, geo_batch.cu)
// Version-1 files ("dtype op conn height width steps_class K ms") load as
// exact entries of the default shape. Entries written on a different device
// name are ignored when GEOMORPH_TUNE_CACHE is loaded.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "geo_common.cuh"

namespace geo {
namespace {

using TuneKey = std::tuple<int, int, int, int64_t, int64_t, int64_t>;
struct TuneVal {
  int K, variant;
  float ms;
  int K0;  // fastest K of the default shape (0: not measured)
  float ms0;
  double work;  // class entries: pixel-steps of the item that set it
};

std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_exact, g_class;
// the batch planner's per-pass charge (geo_batch_autotune); 0: untuned
double g_batch_sync = 0;
float g_batch_ms = 0;

int64_t steps_class(int op, int64_t steps) {
  if (op == 2 || op == 3) return -1;
  return steps < 64 ? steps : 64;
}

int64_t size_class(int64_t n) { return n <= 1 ? 0 : (int64_t)std::floor(2.0 * std::log2((double)n)); }

TuneKey exact_key(int dt, int op, int conn, int64_t H, int64_t W, int64_t steps) {
  return TuneKey{dt, op, conn, H, W, steps_class(op, steps)};
}
TuneKey class_key(int dt, int op, int conn, int64_t H, int64_t W, int64_t steps) {
  return TuneKey{dt, op, conn, size_class(H), size_class(W), steps_class(op, steps)};
}

std::string device_name() {
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string s(p.name);
  for (char &c : s)
    if (c == ' ' || c == '\t') c = '_';
  return s;
}

int load_file(const char *path, bool check_device) {
  FILE *f = fopen(path, "r");
  if (!f) return GEO_ERR_ARG;
  char line[512];
  if (!fgets(line, sizeof line, f)) {
    fclose(f);
    return GEO_ERR_ARG;
  }
  char magic[64] = {0}, dev[256] = {0};
  int ver = 0;
  if (sscanf(line, "%63s %d %255s", magic, &ver, dev) < 2 || strcmp(magic, "geomorph-tune") != 0 ||
      (ver != 1 && ver != 2)) {
    fclose(f);
    return GEO_ERR_ARG;
  }
  if (check_device && dev[0] && device_name() != dev) {
    fclose(f);
    return GEO_OK;  // tuned elsewhere: ignore
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  while (fgets(line, sizeof line, f)) {
    int dt, op, conn, K, v = 0, K0 = 0;
    long long a, b, sc;
    float ms = 0.f, ms0 = 0.f;
    double work = 0;
    char kind = 0;
    if (ver == 1) {
      if (sscanf(line, "%d %d %d %lld %lld %lld %d %f", &dt, &op, &conn, &a, &b, &sc, &K, &ms) >= 7 && K > 0)
        g_exact[TuneKey{dt, op, conn, a, b, sc}] = TuneVal{K, 0, ms, K, ms, 0};
      continue;
    }
    double bs = 0;
    if (sscanf(line, " B %lf %f", &bs, &ms) >= 1) {
      if (bs > 0) {
        g_batch_sync = bs;
        g_batch_ms = ms;
      }
      continue;
    }
    const int n = sscanf(line, " %c %d %d %d %lld %lld %lld %d %d %f %d %f %lf", &kind, &dt, &op, &conn, &a, &b, &sc,
                         &K, &v, &ms, &K0, &ms0, &work);
    if (n < 12 || K <= 0 || v < 0 || v >= kRRVariants) continue;
    const TuneVal val{K, v, ms, K0, ms0, n >= 13 ? work : 0};
    if (kind == 'E') g_exact[TuneKey{dt, op, conn, a, b, sc}] = val;
    if (kind == 'C') g_class[TuneKey{dt, op, conn, a, b, sc}] = val;
  }
  fclose(f);
  return GEO_OK;
}

std::once_flag g_env_once;

// GEOMORPH_TUNE_CACHE is read on first use (outside g_tune_mu: load_file
// takes it itself)
void load_env_once() {
  std::call_once(g_env_once, [] {
    if (const char *p = getenv("GEOMORPH_TUNE_CACHE")) load_file(p, true);
  });
}

int write_file(const char *path) {
  FILE *f = fopen(path, "w");
  if (!f) return GEO_ERR_ARG;
  fprintf(f, "geomorph-tune 2 %s\n", device_name().c_str());
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (int pass = 0; pass < 2; ++pass) {
    for (const auto &kv : pass == 0 ? g_exact : g_class) {
      const TuneKey &k = kv.first;
      const TuneVal &v = kv.second;
      fprintf(f, "%c %d %d %d %lld %lld %lld %d %d %.4f %d %.4f %.0f\n", pass == 0 ? 'E' : 'C', std::get<0>(k),
              std::get<1>(k), std::get<2>(k), (long long)std::get<3>(k), (long long)std::get<4>(k),
              (long long)std::get<5>(k), v.K, v.variant, v.ms, v.K0, v.ms0, v.work);
    }
  }
  if (g_batch_sync > 0) fprintf(f, "B %.4f %.4f\n", g_batch_sync, g_batch_ms);
  fclose(f);
  return GEO_OK;
}

// exact entry, else class entry; nullptr if neither (caller holds g_tune_mu)
const TuneVal *lookup(int dt, int op, int conn, int64_t H, int64_t W, int64_t steps) {
  auto it = g_exact.find(exact_key(dt, op, conn, H, W, steps));
  if (it != g_exact.end()) return &it->second;
  auto jt = g_class.find(class_key(dt, op, conn, H, W, steps));
  if (jt != g_class.end()) return &jt->second;
  return nullptr;
}

}  // namespace

int tuned_k(int dt, int op, int conn, int64_t H, int64_t W, int64_t steps) {
  load_env_once();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const TuneVal *v = lookup(dt, op, conn, H, W, steps);
  return v ? v->K0 : 0;
}

bool tuned_plan(int dt, int op, int conn, int64_t H, int64_t W, int64_t steps, int *K, int *variant) {
  load_env_once();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const TuneVal *v = lookup(dt, op, conn, H, W, steps);
  if (!v) return false;
  *K = v->K;
  *variant = v->variant;
  return true;
}

double tuned_batch_sync() {
  load_env_once();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_batch_sync > 0 ? g_batch_sync : 10.0;
}

void set_tuned_batch_sync(double sync, float ms) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_batch_sync = sync;
  g_batch_ms = ms;
}

}  // namespace geo

using namespace geo;

namespace {

// Time one item with K and the shape variant forced through the calling
// thread's planner override; returns ms per run.
float time_item(const geo_item &x, int K, int variant, int reps, cudaStream_t s, int *rc_out) {
  plan_override() = PlanOverride{K, variant};
  auto once = [&]() -> int {
    switch (x.op) {
      case 0: return geo_dilate_chain(x.dtype, x.marker, x.mask, x.out, x.height, x.width, x.pitch, x.conn, x.steps, s);
      case 1: return geo_erode_chain(x.dtype, x.marker, x.mask, x.out, x.height, x.width, x.pitch, x.conn, x.steps, s);
      case 2:
      case 3:
        return geo_reconstruct(x.dtype, x.marker, x.mask, x.out, x.height, x.width, x.pitch, x.conn, x.op - 2,
                               x.steps, nullptr, s);
      case 4: return morph_window_dilate(x.dtype, x.marker, x.out, x.height, x.width, x.pitch, x.steps, s);
      default: return morph_window_erode(x.dtype, x.marker, x.out, x.height, x.width, x.pitch, x.steps, s);
    }
  };
  int rc = once();  // warm-up (also plans with this K)
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps && rc == GEO_OK; ++r) rc = once();
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  plan_override() = PlanOverride{0, -1};
  *rc_out = rc;
  return reps > 0 ? ms / reps : ms;
}

}  // namespace

extern "C" {

int geo_autotune(const geo_item *items, int n, const char *cache_path) {
  if (n < 0 || (n > 0 && !items)) return GEO_ERR_ARG;
  // a global override would defeat the measurement
  if (getenv("GEOMORPH_K") || getenv("GEOMORPH_VARIANT")) return GEO_ERR_ARG;
  // the items' inputs may still be in flight on other streams
  if (cudaDeviceSynchronize() != cudaSuccess) return GEO_ERR_CUDA;
  cudaStream_t s = nullptr;
  for (int i = 0; i < n; ++i) {
    const geo_item &x = items[i];
    if (x.height <= 0 || x.width <= 0 || x.op < 0 || x.op > 5) continue;
    const int CW = x.dtype == GEO_F64 ? 2 : 4;
    const int nvar = (x.dtype == GEO_U8 || x.dtype == GEO_F32) ? kRRVariants : 1;
    // candidates: multiples of CW up to a third of the register region's
    // longer side (the planner rejects those past the shorter side's third)
    const int kmax = x.dtype == GEO_F64 ? 20 : 40;
    TuneVal best{0, 0, 1e30f, 0, 1e30f, 0};
    for (int v = 0; v < nvar; ++v) {
      for (int K = CW; K <= kmax; K += CW) {
        int rc = GEO_OK;
        const float ms = time_item(x, K, v, 3, s, &rc);
        if (rc != GEO_OK) continue;  // K outside this shape's valid range
        if (ms < best.ms) {
          best.ms = ms;
          best.K = K;
          best.variant = v;
        }
        if (v == 0 && ms < best.ms0) {
          best.ms0 = ms;
          best.K0 = K;
        }
      }
    }
    if (best.K > 0) {
      const int conn = x.op >= 4 ? 8 : x.conn;
      best.work = (double)x.height * (double)x.width *
                  (double)(x.op == 2 || x.op == 3 ? (x.height > x.width ? x.height : x.width) : x.steps + 1);
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_exact[exact_key(x.dtype, x.op, conn, x.height, x.width, x.steps)] = best;
      const TuneKey ck = class_key(x.dtype, x.op, conn, x.height, x.width, x.steps);
      auto it = g_class.find(ck);
      if (it == g_class.end() || it->second.work <= best.work) g_class[ck] = best;
    }
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return GEO_ERR_CUDA;
  if (cache_path && cache_path[0]) return write_file(cache_path);
  return GEO_OK;
}

int geo_tune_load(const char *cache_path) {
  if (!cache_path) return GEO_ERR_ARG;
  return load_file(cache_path, false);
}

int geo_tune_reset(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_exact.clear();
  g_class.clear();
  g_batch_sync = 0;
  g_batch_ms = 0;
  return GEO_OK;
}

int geo_tune_save(const char *cache_path) {
  if (!cache_path) return GEO_ERR_ARG;
  return write_file(cache_path);
}

int geo_tune_lookup(int dtype, int op, int conn, int64_t height, int64_t width, int64_t steps) {
  return tuned_k(dtype, op, conn, height, width, steps);
}

}  // extern "C"
