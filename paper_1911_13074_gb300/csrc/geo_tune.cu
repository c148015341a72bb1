// Measured choice of the pass length K (the halo, which fixes the tile
// interior) per (element type, operation, connectivity, image size, chain
// length class), persisted in a small text file.
//
// The planners first look here and fall back to their cost model. The file
// is text: a header line "geomorph-tune 1 <device name>" and one entry per
// line "dtype op conn height width steps_class K ms". Entries written on a
// different device name are ignored when the file is loaded. steps_class is
// the chain length when it is below 64 (there K may exceed the length) and 64
// otherwise; reconstructions use -1.
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
  int K;
  float ms;
};

std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

int64_t steps_class(int op, int64_t steps) {
  if (op == 2 || op == 3) return -1;
  return steps < 64 ? steps : 64;
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
  int rc = GEO_OK;
  if (!fgets(line, sizeof line, f)) {
    fclose(f);
    return GEO_ERR_ARG;
  }
  char magic[64] = {0}, dev[256] = {0};
  int ver = 0;
  if (sscanf(line, "%63s %d %255s", magic, &ver, dev) < 2 || strcmp(magic, "geomorph-tune") != 0 || ver != 1) {
    fclose(f);
    return GEO_ERR_ARG;
  }
  if (check_device && dev[0] && device_name() != dev) {
    fclose(f);
    return GEO_OK;  // tuned elsewhere: ignore
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  while (fgets(line, sizeof line, f)) {
    int dt, op, conn, K;
    long long H, W, sc;
    float ms = 0.f;
    if (sscanf(line, "%d %d %d %lld %lld %lld %d %f", &dt, &op, &conn, &H, &W, &sc, &K, &ms) >= 7 && K > 0)
      g_tune[TuneKey{dt, op, conn, H, W, sc}] = TuneVal{K, ms};
  }
  fclose(f);
  return rc;
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
  fprintf(f, "geomorph-tune 1 %s\n", device_name().c_str());
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto &kv : g_tune) {
    const TuneKey &k = kv.first;
    fprintf(f, "%d %d %d %lld %lld %lld %d %.4f\n", std::get<0>(k), std::get<1>(k), std::get<2>(k),
            (long long)std::get<3>(k), (long long)std::get<4>(k), (long long)std::get<5>(k), kv.second.K,
            kv.second.ms);
  }
  fclose(f);
  return GEO_OK;
}

}  // namespace

int tuned_k(int dt, int op, int conn, int64_t H, int64_t W, int64_t steps) {
  load_env_once();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(TuneKey{dt, op, conn, H, W, steps_class(op, steps)});
  return it == g_tune.end() ? 0 : it->second.K;
}

}  // namespace geo

using namespace geo;

namespace {

int item_chain_op(const geo_item &x) { return x.op; }

// Time one item with K forced through the planner override; returns ms.
float time_item(const geo_item &x, int K, int reps, cudaStream_t s, int *rc_out) {
  char kbuf[32];
  snprintf(kbuf, sizeof kbuf, "%d", K);
  setenv("GEOMORPH_K", kbuf, 1);
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
  unsetenv("GEOMORPH_K");
  *rc_out = rc;
  return reps > 0 ? ms / reps : ms;
}

}  // namespace

extern "C" {

int geo_autotune(const geo_item *items, int n, const char *cache_path) {
  if (n < 0 || (n > 0 && !items)) return GEO_ERR_ARG;
  if (getenv("GEOMORPH_K")) return GEO_ERR_ARG;  // a global override would defeat the measurement
  // the items' inputs may still be in flight on other streams
  if (cudaDeviceSynchronize() != cudaSuccess) return GEO_ERR_CUDA;
  cudaStream_t s = nullptr;
  for (int i = 0; i < n; ++i) {
    const geo_item &x = items[i];
    if (x.height <= 0 || x.width <= 0 || x.op < 0 || x.op > 5) continue;
    const int CW = x.dtype == GEO_F64 ? 2 : 4;
    // candidates: multiples of CW up to a third of the register region side
    const int kmax = x.dtype == GEO_F64 ? 20 : 40;
    int bestK = 0;
    float best = 1e30f;
    for (int K = CW; K <= kmax; K += CW) {
      int rc = GEO_OK;
      const float ms = time_item(x, K, 3, s, &rc);
      if (rc != GEO_OK) continue;  // K outside this size's valid range
      if (ms < best) {
        best = ms;
        bestK = K;
      }
    }
    if (bestK > 0) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[TuneKey{(int)x.dtype, item_chain_op(x), x.op >= 4 ? 8 : x.conn, x.height, x.width,
                     steps_class(x.op, x.steps)}] = TuneVal{bestK, best};
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

int geo_tune_lookup(int dtype, int op, int conn, int64_t height, int64_t width, int64_t steps) {
  return tuned_k(dtype, op, conn, height, width, steps);
}

}  // extern "C"
