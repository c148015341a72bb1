// Batched geodesic chains: many independent items (uneven sizes, element
// types, operations, lengths, to-stability or fixed) in one persistent,
// cooperative launch fed by a device-side tile work-queue. The paper has no
// batched form; each item computes exactly what its single-item entry point
// computes (Eq. 3-5, or Eq. 1-2 for windows).
//
// Scheduling. A task is one tile of one item for that item's current pass.
// All pass-0 tasks are queued by the init kernel, largest items first. A CTA
// takes the next ticket from the queue head, runs K (or fewer) steps of that
// tile in registers (the register-resident step of geo_rr.cuh) and stores the
// interior. The CTA that completes the last tile of an item's pass decides
// what comes next for that item (another pass, or done: a chain after its
// last pass, a reconstruction after a pass that changed nothing) and pushes
// the item's tiles for the next pass. Items therefore advance independently,
// with no grid-wide barrier; every wait (for a ticket to be filled) is
// bounded and ends when all items are done.
#include <algorithm>
#include <cstring>
#include <vector>

#include "geo_rr.cuh"

namespace geo {

struct BItem {
  Plane marker, mask, out, scratch;
  int64_t H, W;
  int64_t steps;  // chain: steps; reconstruction: max steps
  int dtype, op, conn, rec, alias;
  int K, TH, TW, tiles_x, tiles_y, npasses;
};

struct BState {
  int pass;
  int remaining;  // tiles of the current pass not yet finished
  int changed[2];
  int64_t steps_done;
};

struct BQueue {
  unsigned long long head, tail;
  int items_done;
  int done;
  int pad[2];
};

struct BatchArgs {
  BItem *items;
  BState *state;
  BQueue *q;
  unsigned long long *seq;  // per slot: ticket + 1 once the slot holds that ticket's task
  unsigned long long *task;  // per slot: item << 32 | tile
  unsigned long long cap;
  int n;
  int *status_out;  // per item (device), optional
  int *dev_status;  // sticky per-device status word
};

namespace {

constexpr int kBatchNW = 16;  // warps per CTA, the same for every element policy
static_assert(RU8<0>::NW == kBatchNW && RF32<0>::NW == kBatchNW && RF64<0>::NW == kBatchNW,
              "the batch kernel runs every element policy with one block size");

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Steps of pass p of item it.
__device__ __forceinline__ int pass_steps(const BItem &it, int p, int64_t steps_done) {
  if (!it.rec) {
    const int64_t base = it.steps / it.npasses, extra = it.steps % it.npasses;
    return (int)(base + (p < extra ? 1 : 0));
  }
  const int64_t left = it.steps - steps_done;
  return (int)(left < (int64_t)it.K ? left : (int64_t)it.K);
}

// One tile of one pass with element policy P: load, S steps, store.
template <class P, int CONN>
__device__ bool run_tile(const BItem &it, int tile, int p, int S, typename P::Wd *xb, uint64_t *bars,
                         int &parity) {
  using R = RR<P>;
  using Wd = typename P::Wd;
  constexpr int CW = R::CW, RW = R::RW, PH = R::PH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool to_out = it.rec ? (((p + it.alias) & 1) == 0) : (((it.npasses - 1 - p) & 1) == 0);
  const Plane dst = to_out ? it.out : it.scratch;
  const Plane src = (p == 0) ? it.marker : (to_out ? it.scratch : it.out);
  const bool src_cg = (p > 0) || (it.marker.ptr == it.out.ptr);
  const int ty = tile / it.tiles_x, tx = tile - ty * it.tiles_x;
  const int64_t ty0 = (int64_t)ty * it.TH, tx0 = (int64_t)tx * it.TW;
  const int64_t gy0 = ty0 - it.K + warp * PH;
  const int64_t gx = tx0 - it.K + lane * CW;
  Wd w[RW][CW], m[RW][CW];
  R::template load_words<false>(src, it.H, it.W, gy0, gx, src_cg, false, w);
  R::template load_words<false>(it.mask, it.H, it.W, gy0, gx, false, it.mask.ptr == nullptr, m);
  bool ok = true;
  for (int j = 0; j < S; ++j) {
    ok &= R::template step<CONN>(w, m, xb + (size_t)parity * (kBatchNW + 2) * 2 * R::RWID, bars, parity, lane, warp);
    parity ^= 1;
  }
  const bool changed = R::store(w, dst, src, it.rec != 0, it.H, it.W, ty0, tx0, it.K, it.TH, it.TW, lane, warp);
  return changed || !ok;
}

template <class P>
__device__ bool dispatch_conn(const BItem &it, int tile, int p, int S, char *xb, uint64_t *bars, int &parity) {
  using Wd = typename P::Wd;
  if (it.conn == 8) return run_tile<P, 8>(it, tile, p, S, reinterpret_cast<Wd *>(xb), bars, parity);
  return run_tile<P, 4>(it, tile, p, S, reinterpret_cast<Wd *>(xb), bars, parity);
}

__device__ bool dispatch(const BItem &it, int tile, int p, int S, char *xb, uint64_t *bars, int &parity) {
  if (it.dtype == GEO_U8)
    return it.op == DILATE ? dispatch_conn<RU8<DILATE>>(it, tile, p, S, xb, bars, parity)
                           : dispatch_conn<RU8<ERODE>>(it, tile, p, S, xb, bars, parity);
  if (it.dtype == GEO_F32)
    return it.op == DILATE ? dispatch_conn<RF32<DILATE>>(it, tile, p, S, xb, bars, parity)
                           : dispatch_conn<RF32<ERODE>>(it, tile, p, S, xb, bars, parity);
  return it.op == DILATE ? dispatch_conn<RF64<DILATE>>(it, tile, p, S, xb, bars, parity)
                         : dispatch_conn<RF64<ERODE>>(it, tile, p, S, xb, bars, parity);
}

// identity words for the slots above warp 0 / below the last warp
__device__ void fill_identity_slots(const BItem &it, char *xb) {
  constexpr size_t slot_b = (size_t)2 * 128 * 4;  // two rows of 128 words of 4 bytes (= 64 words of 8)
  const size_t par_b = (size_t)(kBatchNW + 2) * slot_b;
  for (int i = threadIdx.x; i < 2 * 2 * 128; i += blockDim.x) {
    const int par = i / (2 * 128), k = i % (2 * 128);
    uint32_t *top = reinterpret_cast<uint32_t *>(xb + par * par_b);
    uint32_t *bot = reinterpret_cast<uint32_t *>(xb + par * par_b + (size_t)(kBatchNW + 1) * slot_b);
    uint32_t v;
    if (it.dtype == GEO_U8) {
      v = it.op == DILATE ? 0u : 0x00ff00ffu;
    } else if (it.dtype == GEO_F32) {
      v = it.op == DILATE ? 0xff800000u : 0x7f800000u;  // -inf / +inf
    } else {
      // int64 keys: lowest 0x8000000000000000 / highest 0x7fffffffffffffff, little-endian halves
      v = (k & 1) ? (it.op == DILATE ? 0x80000000u : 0x7fffffffu) : (it.op == DILATE ? 0u : 0xffffffffu);
    }
    top[k] = v;
    bot[k] = v;
  }
}

}  // namespace

__global__ void batch_init(BatchArgs A, const int *order) {
  // states, status, queue slots, and the pass-0 tasks in `order`; the
  // pass-0 task count comes from the uploaded item table (whatever policy
  // prepared it)
  __shared__ unsigned long long ntasks0_s;
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int i = 0; i < A.n; ++i) t += (unsigned long long)A.items[i].tiles_x * (unsigned long long)A.items[i].tiles_y;
    ntasks0_s = t;
  }
  __syncthreads();
  const unsigned long long ntasks0 = ntasks0_s;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x) {
    BState s;
    s.pass = 0;
    s.remaining = A.items[i].tiles_x * A.items[i].tiles_y;
    s.changed[0] = s.changed[1] = 0;
    s.steps_done = 0;
    A.state[i] = s;
    // an empty item is complete; the others are overwritten when they complete
    if (A.status_out) A.status_out[i] = s.remaining == 0 ? GEO_OK : GEO_ERR_TIMEOUT;
  }
  // slots past the pass-0 tasks start empty; the first ntasks0 slots are
  // written below by one thread (disjoint ranges, so no ordering is needed)
  for (unsigned long long k = ntasks0 + blockIdx.x * blockDim.x + threadIdx.x; k < A.cap;
       k += (unsigned long long)gridDim.x * blockDim.x)
    A.seq[k] = 0;
  // pass-0 tasks: order[] lists items largest first; expand to tiles
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long t = 0;
    int empty = 0;
    for (int j = 0; j < A.n; ++j) {
      const int i = order[j];
      const int nt = A.items[i].tiles_x * A.items[i].tiles_y;
      if (nt == 0) ++empty;
      for (int k = 0; k < nt; ++k, ++t) {
        A.task[t] = ((unsigned long long)i << 32) | (unsigned)k;
        A.seq[t] = t + 1;
      }
    }
    A.q->head = 0;
    A.q->tail = t;
    A.q->items_done = empty;
    A.q->done = (empty == A.n);
  }
}

__global__ void __launch_bounds__(kBatchNW * 32, 1) batch_kernel(BatchArgs A) {
  __shared__ __align__(16) char xb[2 * (kBatchNW + 2) * 2 * 128 * 4];
  __shared__ __align__(8) uint64_t xbar;  // split-phase step barrier of the whole CTA
  __shared__ unsigned long long task_s;
  __shared__ int flag_s, push_s, next_s, pass_s;
  __shared__ int64_t sdone_s;
  __shared__ BItem it_s;
  if (threadIdx.x == 0) mbar_init(&xbar, kBatchNW * 32);
  __syncthreads();
  int parity = 0;  // parity of the steps done by this CTA: exchange buffer and barrier phase
  const unsigned long long NONE = ~0ull;
  for (;;) {
    if (threadIdx.x == 0) {
      unsigned long long got = NONE;
      const unsigned long long ticket = atomicAdd(&A.q->head, 1ull);
      const unsigned long long slot = ticket % A.cap;
      const unsigned long long t0 = globaltimer_ns();
      unsigned spins = 0;
      for (;;) {
        if (ld_acquire_u64(&A.seq[slot]) == ticket + 1) {
          got = A.task[slot];
          break;
        }
        if (*(volatile int *)&A.q->done) break;
        if ((++spins & 255u) == 0 && globaltimer_ns() - t0 > kWaitLimitNs) {
          record_status(A.dev_status, GEO_ERR_TIMEOUT);
          *(volatile int *)&A.q->done = 1;
          break;
        }
      }
      task_s = got;
    }
    __syncthreads();
    const unsigned long long task = task_s;
    if (task == NONE) break;
    const int i = (int)(task >> 32), tile = (int)(task & 0xffffffffu);
    if (threadIdx.x == 0) {
      it_s = A.items[i];
      pass_s = *(volatile int *)&A.state[i].pass;
      sdone_s = *(volatile int64_t *)&A.state[i].steps_done;
    }
    __syncthreads();
    const BItem &it = it_s;
    const int p = pass_s;
    const int64_t done_steps = sdone_s;
    const int S = pass_steps(it, p, done_steps);
    fill_identity_slots(it, xb);
    __syncthreads();
    if (threadIdx.x == 0) flag_s = 0;
    __syncthreads();
    const bool ch = dispatch(it, tile, p, S, xb, &xbar, parity);
    if (ch) flag_s = 1;
    __syncthreads();
    // completion of this tile; the last tile of the pass schedules the next
    if (threadIdx.x == 0) {
      if (flag_s) atomicOr(&A.state[i].changed[p & 1], 1);
      __threadfence();
      const int left = atomicSub(&A.state[i].remaining, 1) - 1;
      push_s = 0;
      if (left == 0) {
        __threadfence();
        const int changed = *(volatile int *)&A.state[i].changed[p & 1];
        const int64_t sd = done_steps + S;
        bool more;
        if (!it.rec) {
          more = (p + 1 < it.npasses);
        } else {
          more = changed && sd < it.steps;
          if (!more && A.status_out) A.status_out[i] = changed ? GEO_ERR_NOT_CONVERGED : GEO_OK;
        }
        if (!it.rec && !more && A.status_out) A.status_out[i] = GEO_OK;
        if (more) {
          BState &st = A.state[i];
          st.changed[(p + 1) & 1] = 0;
          st.steps_done = sd;
          st.remaining = it.tiles_x * it.tiles_y;
          st.pass = p + 1;
          __threadfence();
          push_s = it.tiles_x * it.tiles_y;
          next_s = i;
        } else {
          __threadfence();
          if (atomicAdd(&A.q->items_done, 1) + 1 == A.n) {
            __threadfence();
            *(volatile int *)&A.q->done = 1;
          }
        }
      }
    }
    __syncthreads();
    if (push_s > 0) {
      // push the item's tiles for its next pass, using the whole CTA
      __shared__ unsigned long long base_s;
      if (threadIdx.x == 0) base_s = atomicAdd(&A.q->tail, (unsigned long long)push_s);
      __syncthreads();
      const unsigned long long base = base_s;
      for (int k = threadIdx.x; k < push_s; k += blockDim.x) {
        const unsigned long long t = base + k, slot = t % A.cap;
        A.task[slot] = ((unsigned long long)next_s << 32) | (unsigned)k;
        __threadfence();
        st_release_u64(&A.seq[slot], t + 1);
      }
      __syncthreads();
    }
  }
}

}  // namespace geo

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

using namespace geo;

namespace {

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

int elem_bytes(int dt) { return dt == GEO_U8 ? 1 : dt == GEO_F32 ? 4 : 8; }

struct RRG {
  int CW, RW, NW, B;
};
RRG rrg(int dt) {
  if (dt == GEO_U8) return RRG{RU8<0>::CW, RU8<0>::RW, RU8<0>::NW, RU8<0>::BANDS};
  if (dt == GEO_F32) return RRG{RF32<0>::CW, RF32<0>::RW, RF32<0>::NW, RF32<0>::BANDS};
  return RRG{RF64<0>::CW, RF64<0>::RW, RF64<0>::NW, RF64<0>::BANDS};
}

bool is_rec(const geo_item &x) { return x.op == 2 || x.op == 3; }
bool is_win(const geo_item &x) { return x.op == 4 || x.op == 5; }
bool is_empty(const geo_item &x) { return x.height == 0 || x.width == 0; }

// Candidate per-pass charges of the batch planner's cost model (the policy
// geo_batch_autotune chooses among; 10 is the untuned default).
constexpr double kBatchSyncs[] = {2.5, 5.0, 10.0, 20.0, 40.0, 80.0};
constexpr int kNumBatchSyncs = sizeof(kBatchSyncs) / sizeof(kBatchSyncs[0]);

// K for one item: the register-resident region of its element type with the
// halo chosen by a cost model for tiles that run concurrently with other
// items' tiles: tile-steps plus `sync` region-steps per pass (the pass
// hand-over and the queue). The single-image tune entries are not used
// here: they favour many tiles, which a batch does not need (it gets its
// parallelism from the other items). GEOMORPH_BATCH_K overrides K.
int item_k(const geo_item &x, double sync) {
  const RRG g = rrg(x.dtype);
  const int RWID = 32 * g.CW, RHGT = g.NW * g.RW * g.B;
  const int kmax = (RWID < RHGT ? RWID : RHGT) / 2 - g.CW;
  if (const char *e = getenv("GEOMORPH_BATCH_K")) {
    int k = ((atoi(e) + g.CW - 1) / g.CW) * g.CW;
    if (k >= g.CW && k <= kmax) return k;
  }
  const bool rec = is_rec(x);
  double best = 1e300;
  int bk = g.CW;
  const double n = rec ? (double)(x.height > x.width ? x.height : x.width) : (double)(x.steps > 0 ? x.steps : 1);
  for (int K = g.CW; K <= kmax; K += g.CW) {
    const int TW = RWID - 2 * K, TH = RHGT - 2 * K;
    const double tiles = (double)((x.height + TH - 1) / TH) * (double)((x.width + TW - 1) / TW);
    const double passes = rec ? (n / K + 2.0) : (double)((int64_t)((n + K - 1) / K));
    const double cost = tiles * (passes * sync + (rec ? n + 1.5 * K : n));
    if (cost < best) {
      best = cost;
      bk = K;
    }
  }
  return bk;
}

bool item_valid(const geo_item &x) {
  if (x.op < 0 || x.op > 5) return false;
  if (x.dtype != GEO_U8 && x.dtype != GEO_F32 && x.dtype != GEO_F64) return false;
  if (x.height < 0 || x.width < 0 || x.pitch < x.width) return false;
  if (!is_win(x) && x.conn != 4 && x.conn != 8) return false;
  if (is_empty(x)) return true;
  if (!x.marker || !x.out) return false;
  if (!is_win(x) && !x.mask) return false;
  if (!is_rec(x) && x.steps < 0) return false;
  const int es = elem_bytes(x.dtype);
  if ((uintptr_t)x.marker % es || (uintptr_t)x.out % es || (x.mask && (uintptr_t)x.mask % es)) return false;
  // out may alias marker; it must not overlap the mask
  const size_t span = (size_t)((x.height - 1) * x.pitch * es + x.width * es);
  auto ov = [&](const void *a, const void *b) {
    const char *p = (const char *)a, *q = (const char *)b;
    return p < q + span && q < p + span;
  };
  if (!is_win(x) && ov(x.mask, x.out)) return false;
  if (x.marker != x.out && ov(x.marker, x.out)) return false;
  return true;
}

struct Geometry {
  int K, TH, TW, tiles_x, tiles_y;
};

Geometry item_geometry(const geo_item &x, double sync) {
  Geometry g{};
  if (is_empty(x)) return g;
  const RRG r = rrg(x.dtype);
  g.K = item_k(x, sync);
  g.TW = 32 * r.CW - 2 * g.K;
  g.TH = r.NW * r.RW * r.B - 2 * g.K;
  g.tiles_x = (int)((x.width + g.TW - 1) / g.TW);
  g.tiles_y = (int)((x.height + g.TH - 1) / g.TH);
  return g;
}

struct BatchLayout {
  size_t off_items, off_state, off_q, off_seq, off_task, off_order, off_scratch, total;
  unsigned long long cap;
  std::vector<Geometry> geom;
  std::vector<size_t> scratch_off;
};

// The layout holds the geometry of the policy `sync`; its offsets and queue
// capacity are the same for every candidate policy (the capacity covers the
// most tiles any of them plans), so that a workspace sized once serves every
// policy and geo_batch_launch need not know which one prepared it.
BatchLayout batch_layout(const geo_item *items, int n, double sync) {
  BatchLayout L;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  size_t off = 0;
  L.off_items = off;
  off += up256(sizeof(BItem) * nn);
  L.off_state = off;
  off += up256(sizeof(BState) * nn);
  L.off_q = off;
  off += up256(sizeof(BQueue));
  unsigned long long tiles = 0;
  L.geom.resize(n);
  for (int i = 0; i < n; ++i) L.geom[i] = item_geometry(items[i], sync);
  for (int c = 0; c < kNumBatchSyncs; ++c) {
    unsigned long long t = 0;
    for (int i = 0; i < n; ++i) {
      const Geometry g = item_geometry(items[i], kBatchSyncs[c]);
      t += (unsigned long long)g.tiles_x * (unsigned long long)g.tiles_y;
    }
    if (t > tiles) tiles = t;
  }
  L.cap = 2 * tiles + 64;
  L.off_seq = off;
  off += up256(sizeof(unsigned long long) * L.cap);
  L.off_task = off;
  off += up256(sizeof(unsigned long long) * L.cap);
  L.off_order = off;
  off += up256(sizeof(int) * nn);
  L.off_scratch = off;
  L.scratch_off.resize(n);
  for (int i = 0; i < n; ++i) {
    L.scratch_off[i] = off;
    const geo_item &x = items[i];
    if (!is_empty(x))
      off += up256((size_t)(((x.width * elem_bytes(x.dtype) + 15) / 16) * 16) * (size_t)x.height);
  }
  L.total = off;
  return L;
}

BatchArgs batch_args(const BatchLayout &L, int n, void *workspace, int *status_out, int *dev_status) {
  char *base = (char *)workspace;
  BatchArgs A;
  A.items = (BItem *)(base + L.off_items);
  A.state = (BState *)(base + L.off_state);
  A.q = (BQueue *)(base + L.off_q);
  A.seq = (unsigned long long *)(base + L.off_seq);
  A.task = (unsigned long long *)(base + L.off_task);
  A.cap = L.cap;
  A.n = n;
  A.status_out = status_out;
  A.dev_status = dev_status;
  return A;
}

int check_items(const geo_item *items, int n) {
  if (n < 0 || (n > 0 && !items)) return GEO_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (items[i].dtype != GEO_U8 && items[i].dtype != GEO_F32 && items[i].dtype != GEO_F64) return GEO_ERR_DTYPE;
    if (!item_valid(items[i])) return GEO_ERR_ARG;
  }
  return GEO_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// geo_batch_prepare with the planner's per-pass charge `sync`
int prepare_with(const geo_item *items, int n, void *workspace, size_t ws_bytes, void *stream, double sync) {
  int rc = check_items(items, n);
  if (rc != GEO_OK) return rc;
  if (!workspace) return GEO_ERR_ARG;
  const BatchLayout L = batch_layout(items, n, sync);
  if (ws_bytes < L.total) return GEO_ERR_WORKSPACE;
  // set up the device's library state here (its first use allocates), so
  // that geo_batch_launch allocates nothing and can be captured in a graph
  int *dev_status = nullptr;
  rc = device_status_word(&dev_status);
  if (rc != GEO_OK) return rc;
  std::vector<BItem> table(n);
  std::vector<double> cost(n);
  for (int i = 0; i < n; ++i) {
    const geo_item &x = items[i];
    const Geometry &g = L.geom[i];
    BItem b;
    memset(&b, 0, sizeof(b));
    cost[i] = 0;
    if (!is_empty(x)) {
      const int es = elem_bytes(x.dtype);
      const int64_t pitch_b = x.pitch * es;
      const size_t va = (size_t)rrg(x.dtype).CW * es;
      auto plane = [&](const void *p, int64_t pb) {
        Plane q;
        q.ptr = (char *)p;
        q.pitch_b = pb;
        q.vec_ok = (p != nullptr && ((uintptr_t)p % va) == 0 && pb % (int64_t)va == 0) ? 1 : 0;
        q.bstride = 0;
        return q;
      };
      const bool rec = is_rec(x), win = is_win(x);
      b.marker = plane(x.marker, pitch_b);
      b.mask = win ? plane(nullptr, pitch_b) : plane(x.mask, pitch_b);
      b.out = plane(x.out, pitch_b);
      b.scratch = plane((char *)workspace + L.scratch_off[i], ((x.width * es + 15) / 16) * 16);
      b.H = x.height;
      b.W = x.width;
      b.dtype = x.dtype;
      b.op = (x.op == 1 || x.op == 3 || x.op == 5) ? ERODE : DILATE;
      b.conn = win ? 8 : x.conn;
      b.rec = rec ? 1 : 0;
      b.alias = (x.marker == x.out) ? 1 : 0;
      b.K = g.K;
      b.TH = g.TH;
      b.TW = g.TW;
      b.tiles_x = g.tiles_x;
      b.tiles_y = g.tiles_y;
      if (rec) {
        b.steps = x.steps > 0 ? x.steps : x.height * x.width + 1 + 1024;
      } else {
        b.steps = x.steps;
        int64_t np = (x.steps + g.K - 1) / g.K;
        if (np < 1) np = 1;  // a 0-step item is one pass of 0 steps: a copy
        if (b.alias && (np & 1)) ++np;
        b.npasses = (int)np;
      }
      const double len = rec ? (double)(x.height > x.width ? x.height : x.width) : (double)(x.steps + 1);
      cost[i] = (double)g.tiles_x * (double)g.tiles_y * len;
    }
    table[i] = b;
  }
  std::vector<int> order(n);
  for (int j = 0; j < n; ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  cudaStream_t s = (cudaStream_t)stream;
  char *base = (char *)workspace;
  if (n > 0) {
    // pageable sources: the runtime stages them before returning
    if (cudaMemcpyAsync(base + L.off_items, table.data(), sizeof(BItem) * n, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return GEO_ERR_CUDA;
    if (cudaMemcpyAsync(base + L.off_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return GEO_ERR_CUDA;
  }
  return GEO_OK;
}

}  // namespace

extern "C" {

size_t geo_batch_workspace_size(const geo_item *items, int n) {
  if (check_items(items, n) != GEO_OK) return 0;
  return batch_layout(items, n, kBatchSyncs[0]).total;  // the same for every policy
}

int geo_batch_prepare(const geo_item *items, int n, void *workspace, size_t ws_bytes, void *stream) {
  return prepare_with(items, n, workspace, ws_bytes, stream, tuned_batch_sync());
}

int geo_batch_launch(const geo_item *items, int n, void *workspace, int *status_out, void *stream) {
  int rc = check_items(items, n);
  if (rc != GEO_OK) return rc;
  if (!workspace) return GEO_ERR_ARG;
  if (n == 0) return GEO_OK;
  // offsets and queue capacity only (the same for every policy)
  const BatchLayout L = batch_layout(items, n, kBatchSyncs[0]);
  int *dev_status = nullptr;
  rc = device_status_word(&dev_status);
  if (rc != GEO_OK) return rc;
  BatchArgs A = batch_args(L, n, workspace, status_out, dev_status);
  cudaStream_t s = (cudaStream_t)stream;
  const int *order = (const int *)((char *)workspace + L.off_order);
  batch_init<<<64, 256, 0, s>>>(A, order);
  if (cudaGetLastError() != cudaSuccess) return GEO_ERR_CUDA;
  int dev = 0, nsm = 0, bps = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GEO_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GEO_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, batch_kernel, kBatchNW * 32, 0) != cudaSuccess || bps < 1)
    return GEO_ERR_CUDA;
  int grid = bps * nsm;
  if (const char *e = getenv("GEOMORPH_BATCH_GRID")) {
    const int g = atoi(e);
    if (g > 0 && g < grid) grid = g;
  }
  void *args[] = {(void *)&A};
  if (cudaLaunchCooperativeKernel((void *)batch_kernel, dim3(grid), dim3(kBatchNW * 32), args, 0, s) != cudaSuccess)
    return GEO_ERR_CUDA;
  return GEO_OK;
}

int geo_batch_autotune(const geo_item *items, int n, void *workspace, size_t ws_bytes, int *status_out,
                       void *stream, const char *cache_path) {
  int rc = check_items(items, n);
  if (rc != GEO_OK) return rc;
  if (!workspace || n == 0) return n == 0 ? GEO_OK : GEO_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GEO_ERR_CUDA;
  std::vector<int> st(status_out ? n : 0);
  double best_sync = 0;
  float best_ms = 1e30f;
  for (int c = 0; c < kNumBatchSyncs && rc == GEO_OK; ++c) {
    rc = prepare_with(items, n, workspace, ws_bytes, stream, kBatchSyncs[c]);
    if (rc == GEO_OK) rc = geo_batch_launch(items, n, workspace, status_out, stream);  // warm-up
    if (rc != GEO_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 2 && rc == GEO_OK; ++r) rc = geo_batch_launch(items, n, workspace, status_out, stream);
    cudaEventRecord(e1, s);
    if (rc != GEO_OK || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = rc != GEO_OK ? rc : GEO_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= 2;
    // a policy under which an item did not complete is not a candidate
    bool ok = true;
    if (status_out) {
      if (cudaMemcpy(st.data(), status_out, sizeof(int) * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = GEO_ERR_CUDA;
        break;
      }
      for (int v : st) ok &= (v == GEO_OK || v == GEO_ERR_NOT_CONVERGED);
    }
    if (ok && ms < best_ms) {
      best_ms = ms;
      best_sync = kBatchSyncs[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != GEO_OK) return rc;
  if (best_sync <= 0) return GEO_ERR_CUDA;
  set_tuned_batch_sync(best_sync, best_ms);
  // leave the workspace prepared with the chosen policy
  rc = prepare_with(items, n, workspace, ws_bytes, stream, best_sync);
  if (rc == GEO_OK && cache_path && cache_path[0]) rc = geo_tune_save(cache_path);
  return rc;
}

int geo_batch(const geo_item *items, int n, void *workspace, size_t ws_bytes, int *status_out, void *stream) {
  int rc = geo_batch_prepare(items, n, workspace, ws_bytes, stream);
  if (rc != GEO_OK) return rc;
  return geo_batch_launch(items, n, workspace, status_out, stream);
}

}  // extern "C"
