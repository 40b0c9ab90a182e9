// C ABI of the TSQR library: argument checking, the planner (leaf partition, chains,
// reduction tree), the device-resident plan cache, the factor-set object and the opt-in
// launch profiler. Every public entry point is declared and documented in include/tsqr.h.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <list>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/tsqr.h"
#include "tsqr_internal.h"

using namespace tsqr;

namespace {

// The calling thread's last error message, in a fixed buffer: setting or clearing it
// never allocates (the allocation-free entry point reports through it too).
struct ErrorText {
  char buf[512];
  void clear() { buf[0] = 0; }
  const char *c_str() const { return buf; }
  void vset(const char *fmt, va_list ap) {
    char tmp[sizeof buf];  // the arguments may point into buf
    vsnprintf(tmp, sizeof tmp, fmt, ap);
    memcpy(buf, tmp, sizeof buf);
  }
};
thread_local ErrorText g_last_error = {{0}};

tsqr_status fail(tsqr_status s, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  g_last_error.vset(fmt, ap);
  va_end(ap);
  return s;
}

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? TSQR_ERR_OOM : TSQR_ERR_CUDA,         \
                  "%s failed: %s", #expr, cudaGetErrorString(e_));                        \
  } while (0)

struct DeviceInfo {
  int sms = 0;
  size_t smem_sm = 0, reserved = 0, optin = 0;
};

DeviceInfo device_info(int dev) {
  static std::mutex mu;
  static std::vector<DeviceInfo> cache;
  std::lock_guard<std::mutex> lk(mu);
  if ((int)cache.size() <= dev) cache.resize(dev + 1);
  DeviceInfo &d = cache[dev];
  if (d.sms == 0) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
      d.sms = prop.multiProcessorCount;
      d.smem_sm = prop.sharedMemPerMultiprocessor;
      d.reserved = prop.reservedSharedMemPerBlock;
      d.optin = prop.sharedMemPerBlockOptin;
    }
  }
  return d;
}

// Test hook (tsqr_debug_fail_allocations): the next N device allocations of the library
// fail as if the device were out of memory.
std::atomic<int32_t> g_fail_allocs{0};

// Mixed-precision items with at least this many columns factor their FP32 chains by
// compact-WY panels with 3xTF32 tensor-core updates (0: never; tsqr_set_mixed_wy_min_n).
std::atomic<int32_t> g_wy_min_n{0};

// Q^T b and Q b with one column run the tile-pair kernel on launches whose jobs hold
// several tiles (1, the default; 0: the one-warp-per-tile kernel; tsqr_set_apply_tile_pairs).
std::atomic<int32_t> g_tile_pairs{1};

// Stream-ordered allocations come from a memory pool of the library's own, one per device,
// kept cached so that repeated factorizations do not return memory to the driver. Its
// blocks freed on one stream are not reused by another stream through an inserted
// dependency (cudaMemPoolReuseAllowInternalDependencies off): calls in flight on two
// streams (the server's batches, pipelined host-buffer calls) then take fresh memory
// instead of waiting for the other call's end.
cudaError_t lib_pool(int dev, cudaMemPool_t *out) {
  static std::mutex mu;
  static std::vector<std::pair<int, cudaMemPool_t>> pools;
  std::lock_guard<std::mutex> lk(mu);
  for (auto &dp : pools)
    if (dp.first == dev) {
      *out = dp.second;
      return cudaSuccess;
    }
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool;
  cudaError_t e = cudaMemPoolCreate(&pool, &props);
  if (e != cudaSuccess) return e;
  uint64_t thr = UINT64_MAX;
  int no = 0;
  e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  if (e == cudaSuccess) e = cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
  if (e != cudaSuccess) {
    cudaMemPoolDestroy(pool);
    return e;
  }
  pools.push_back({dev, pool});
  *out = pool;
  return cudaSuccess;
}

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s) {
  if (tsqr::debug_take_allocation_failure()) return cudaErrorMemoryAllocation;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool;
  e = lib_pool(dev, &pool);
  if (e != cudaSuccess) return e;
  if (bytes == 0) bytes = 16;
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

// One non-blocking helper stream per device, for work the library overlaps with the
// caller's stream (joined back with events before the call's later work).
cudaStream_t helper_stream(int dev) {
  static std::mutex mu;
  static std::vector<std::pair<int, cudaStream_t>> streams;
  std::lock_guard<std::mutex> lk(mu);
  for (auto &ds : streams)
    if (ds.first == dev) return ds.second;
  cudaStream_t hs = nullptr;
  if (cudaStreamCreateWithFlags(&hs, cudaStreamNonBlocking) != cudaSuccess) hs = nullptr;
  streams.push_back({dev, hs});
  return hs;
}

// ------------------------------------------------------------------- profiler
// Opt-in: a pair of CUDA events recorded on the launching stream around every kernel
// launch the library makes, read back by tsqr_profile_stop.
struct ProfRec {
  int32_t kind;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;

struct ProfScope {
  bool on = false;
  cudaStream_t s;
  ProfRec r{};
  ProfScope(int32_t kind, cudaStream_t st) : s(st) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on || kind < 0) return;  // kind < 0: never recorded (graph capture)
    r.kind = kind;
    if (cudaEventCreate(&r.a) != cudaSuccess) return;
    if (cudaEventCreate(&r.b) != cudaSuccess) {
      cudaEventDestroy(r.a);
      return;
    }
    cudaEventRecord(r.a, s);
    on = true;
  }
  ~ProfScope() {
    if (!on) return;
    cudaEventRecord(r.b, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.push_back(r);
  }
};

}  // namespace

// ------------------------------------------------------------------------- plan
struct Plan {
  int64_t m = 0;
  int n = 0, nc = 0, leaf_h = 0, arity = 0, flags = 0, tile_h = 0, ctas_per_sm = 0;
  bool mixed = false;  // FP32 chains on global rows, FP64 tree on compact pivot blocks
  int64_t leaves = 0;
  std::vector<TileDesc> tiles;
  std::vector<JobDesc> jobs;
  std::vector<LaunchDesc> launches;  // launch 0: chains; 1..: tree levels
  // TSQR_CLUSTER: the factorization runs binary levels lo..hi of the tree in one launch of
  // clusters (kClusterSize slots per cluster); the apply kernels keep the per-level launches
  struct ClusterLaunch {
    int32_t slot_begin, nclusters, level_lo, level_hi;
  };
  std::vector<ClusterLaunch> cl_launches;
  std::vector<ClusterSlot> cl_slots;
  std::vector<ApplyClusterSlot> cl_apply;  // the same slots seen top down (parents), for Q B
  int cl_base = 0;  // tree levels 1..cl_base run one launch each before the cluster launches
  // factorization launches (the chain launch, the per-level tree launches, the cluster launches)
  int factor_launches() const {
    return cl_launches.empty() ? (int)launches.size() : 1 + cl_base + (int)cl_launches.size();
  }
};

// Groups the binary tree's levels three at a time into cluster launches: cluster c of the
// launch based at level b holds the 8 consecutive nodes 8c..8c+7 of level b (complete in
// global memory) and the combine jobs of levels b+1..b+3 over them. Node i of level t covers
// the base nodes [i 2^(t-b), (i+1) 2^(t-b)) (a lone node passes up only at the end of a
// level), so the groups are exactly subtrees of the binary tree.
//
// Levels wide enough to fill the GPU (more clusters than fit at once: max_ctas CTAs) stay
// one launch per level: there the combines are throughput-bound and a cluster's waiting
// CTAs would only take slots (measured at 4M x 64: 1.60 ms for levels 1-3 as one cluster
// launch of four waves, 1.28 ms as three launches). The cluster launches start at the
// first level whose clusters all fit at once, where the levels are latency-bound.
static void plan_clusters(Plan &pl, int64_t max_ctas) {
  const int L = (int)pl.launches.size() - 1;
  if (L < 1) return;
  std::vector<int64_t> N(L + 1);
  N[0] = pl.launches[0].job_count;
  for (int t = 1; t <= L; ++t) N[t] = (N[t - 1] + 1) / 2;
  int b0 = 0;
  while (b0 < L && (N[b0] + kClusterSize - 1) / kClusterSize * kClusterSize > max_ctas) ++b0;
  if (b0 >= L) return;
  pl.cl_base = b0;
  for (int b = b0; b < L; b += 3) {
    const int top = std::min(L, b + 3);
    const int64_t span = int64_t(1) << (top - b);
    const int64_t ncl = (N[b] + span - 1) / span;
    Plan::ClusterLaunch cl{(int32_t)pl.cl_slots.size(), (int32_t)ncl, b + 1, top};
    for (int64_t c = 0; c < ncl; ++c) {
      ClusterSlot sl[kClusterSize];
      for (auto &x : sl) x = {-1, {-1, -1}, 0};
      int prod[4][kClusterSize];  // cluster rank producing node (level t - b, local index)
      for (int q = 0; q < kClusterSize; ++q) prod[0][q] = -1;
      int rank = 0;
      for (int t = b + 1; t <= top; ++t) {
        const int64_t per = span >> (t - b);
        for (int64_t il = 0; il < per; ++il) {
          const int64_t i = c * per + il;
          if (i >= N[t]) break;
          int *pv = prod[t - b - 1];
          const int64_t l0 = 2 * il;  // local index of node 2i at level t - 1
          if (i < N[t - 1] / 2) {
            sl[rank] = {pl.launches[t].job_begin + (int32_t)i, {pv[l0], pv[l0 + 1]}, 0};
            prod[t - b][il] = rank++;
          } else {
            prod[t - b][il] = pv[l0];  // passes up unchanged
          }
        }
      }
      pl.cl_slots.insert(pl.cl_slots.end(), sl, sl + kClusterSize);
      // top down: each in-cluster child's parent and the side of the parent it continues
      ApplyClusterSlot as[kClusterSize];
      for (int r = 0; r < kClusterSize; ++r) as[r] = {sl[r].job, -1, 0, 0};
      for (int r = 0; r < kClusterSize; ++r)
        for (int q = 0; q < 2; ++q)
          if (sl[r].job >= 0 && sl[r].child[q] >= 0) {
            as[sl[r].child[q]].parent = r;
            as[sl[r].child[q]].side = q;
            as[r].kids |= 1 << q;
          }
      pl.cl_apply.insert(pl.cl_apply.end(), as, as + kClusterSize);
    }
    pl.cl_launches.push_back(cl);
  }
}

static void plan_build(Plan &pl, int64_t chains_target) {
  const int64_t m = pl.m, h = pl.leaf_h;
  const int64_t P = std::max<int64_t>(1, m / h);
  pl.leaves = P;
  auto leaf_begin = [&](int64_t i) { return i * h; };
  auto leaf_end = [&](int64_t i) { return (i == P - 1) ? m : (i + 1) * h; };
  int64_t G;
  if (pl.flags & TSQR_TWO_LEVEL)
    G = std::max<int64_t>(1, std::min<int64_t>(P, chains_target));
  else if (pl.arity == 0)
    G = 1;
  else
    G = P;
  std::vector<int64_t> piv;
  piv.reserve(G);
  pl.launches.push_back({0, 0});
  for (int64_t c = 0; c < G; ++c) {
    const int64_t la = c * P / G, lb = (c + 1) * P / G;  // leaves [la, lb)
    JobDesc job{leaf_begin(la), (int32_t)pl.tiles.size(), 0};
    bool first = true;
    for (int64_t l = la; l < lb; ++l) {
      int64_t r = leaf_begin(l);
      const int64_t r1 = leaf_end(l);
      while (r < r1) {
        const int hh = (int)std::min<int64_t>(pl.tile_h, r1 - r);
        pl.tiles.push_back({r, (int64_t)pl.tiles.size() * pl.n, hh, first ? GEQRT : TSQRT});
        first = false;
        r += hh;
      }
    }
    job.tile_count = (int32_t)pl.tiles.size() - job.tile_begin;
    pl.jobs.push_back(job);
    piv.push_back(job.piv_row);
  }
  pl.launches[0].job_count = (int32_t)pl.jobs.size();
  while (piv.size() > 1) {
    LaunchDesc ld{(int32_t)pl.jobs.size(), 0};
    std::vector<int64_t> next;
    const size_t k = (pl.arity == 0) ? piv.size() : (size_t)pl.arity;
    for (size_t g = 0; g < piv.size(); g += k) {
      const size_t ge = std::min(piv.size(), g + k);
      next.push_back(piv[g]);
      if (ge - g < 2) continue;  // a lone node passes up unchanged
      JobDesc job{piv[g], (int32_t)pl.tiles.size(), 0};
      for (size_t c = g + 1; c < ge; ++c)
        pl.tiles.push_back({piv[c], (int64_t)pl.tiles.size() * pl.n, pl.n, TTQRT});
      job.tile_count = (int32_t)pl.tiles.size() - job.tile_begin;
      pl.jobs.push_back(job);
    }
    ld.job_count = (int32_t)pl.jobs.size() - ld.job_begin;
    pl.launches.push_back(ld);
    piv.swap(next);
  }
}

// Splits every TTQRT tile into pieces of at most h rows of the child's triangle, so that
// a tree node needs no more shared memory than a chain tile (the batched kernel runs
// both in one launch). Reflector indices are renumbered tile by tile. Returns the piece
// height (n when nothing is split).
static int split_tree_tiles(Plan &pl, int h) {
  if (h <= 0 || h >= pl.n) return pl.n;
  const int pieces = (pl.n + h - 1) / h;
  const int ph = (pl.n + pieces - 1) / pieces;
  std::vector<TileDesc> tiles;
  tiles.reserve(pl.tiles.size() * 2);
  for (JobDesc &jd : pl.jobs) {
    const int32_t b = (int32_t)tiles.size();
    for (int32_t t = jd.tile_begin; t < jd.tile_begin + jd.tile_count; ++t) {
      const TileDesc &td = pl.tiles[t];
      if (td.kind != TTQRT) {
        TileDesc c = td;
        c.refl = (int64_t)tiles.size() * pl.n;
        tiles.push_back(c);
        continue;
      }
      for (int o = 0; o < pl.n; o += ph)
        tiles.push_back({td.row0 + o, (int64_t)tiles.size() * pl.n, std::min(ph, pl.n - o), TTQRT, o, 0});
    }
    jd.tile_begin = b;
    jd.tile_count = (int32_t)tiles.size() - b;
  }
  pl.tiles.swap(tiles);
  return ph;
}

// Chooses the tile height and CTAs per SM of the factor kernel for nc columns: two
// resident CTAs when the tile still holds at least n rows (one CTA's scalar phase is
// then hidden behind the other's updates), otherwise one.
// max_cps: the persistent batched kernel is built for two CTAs per SM; the one-problem
// launches may run three.
static bool choose_tiles(const DeviceInfo &di, int n, int nc, int leaf_h, int &tile_h, int &cps,
                         size_t elem = sizeof(double), int max_cps = 3) {
  if (elem == sizeof(float)) {  // register-tile FP32 chains: fixed 128-row tiles
    if (nc > 128) return false;
    tile_h = std::min(kF32TileRows, std::max(leaf_h, n));
    cps = 2;
    return true;
  }
  return factor_tile_choice(n, nc, leaf_h, di.smem_sm, di.reserved, di.optin, max_cps, tile_h, cps);
}

static tsqr_status make_plan_on(const DeviceInfo &di, Plan &pl, int64_t m, int n, int nc, int leaf_h,
                                int arity, int flags, bool mixed = false, int64_t chains_override = 0,
                                int max_cps = 3) {
  pl.m = m;
  pl.n = n;
  pl.nc = nc;
  pl.leaf_h = leaf_h;
  pl.arity = arity;
  pl.flags = flags & (TSQR_TWO_LEVEL | TSQR_CLUSTER);
  pl.mixed = mixed;
  if (!choose_tiles(di, n, nc, leaf_h, pl.tile_h, pl.ctas_per_sm, mixed ? sizeof(float) : sizeof(double), max_cps))
    return fail(TSQR_ERR_UNSUPPORTED, "no tile height fits shared memory for nc=%d", nc);
  // four waves of chains: the apply kernels run one warp per chain, so fewer chains would
  // starve them (the batched path, which applies nothing, sets its own count)
  const int64_t chains = chains_override > 0 ? chains_override : (int64_t)di.sms * pl.ctas_per_sm * 4;
  try {
    plan_build(pl, chains);
    const size_t csm = cluster_smem_bytes(n, nc, di.optin);
    // resident cluster CTAs per SM: the shared-memory limit, and the register limit (288
    // threads per CTA at 64 registers, 80 beyond 64 columns: three, two)
    const int64_t cl_cps = std::min<int64_t>(nc > 64 ? 2 : 3, (int64_t)(di.smem_sm / (csm + di.reserved + 1024)));
    if ((pl.flags & TSQR_CLUSTER) && pl.arity == 2 && !mixed && csm > 0 && cl_cps >= 1)
      plan_clusters(pl, (int64_t)di.sms * cl_cps);
    if (mixed) {
      // the tree works on a compact FP64 array: chain c's pivot block at rows c*n..c*n+n-1
      std::vector<std::pair<int64_t, int64_t>> idx;  // (global pivot row, chain)
      const int32_t G = pl.launches[0].job_count;
      for (int32_t c = 0; c < G; ++c) idx.push_back({pl.jobs[c].piv_row, c});
      std::sort(idx.begin(), idx.end());
      auto compact = [&](int64_t row) {
        auto it = std::lower_bound(idx.begin(), idx.end(), std::make_pair(row, (int64_t)-1));
        return it->second * (int64_t)n;
      };
      for (size_t q = 1; q < pl.launches.size(); ++q) {
        const LaunchDesc &ld = pl.launches[q];
        for (int32_t jb = ld.job_begin; jb < ld.job_begin + ld.job_count; ++jb) {
          JobDesc &jd = pl.jobs[jb];
          for (int32_t t = jd.tile_begin; t < jd.tile_begin + jd.tile_count; ++t)
            pl.tiles[t].row0 = compact(pl.tiles[t].row0);
          jd.piv_row = compact(jd.piv_row);
        }
      }
    }
  } catch (const std::bad_alloc &) {
    return fail(TSQR_ERR_OOM, "host allocation failed while planning");
  }
  return TSQR_OK;
}

// A plan together with its job and tile arrays resident on one device. Plans are
// cached by shape so repeated factorizations of one shape upload nothing.
struct DevPlan {
  Plan plan;
  int device = -1;
  JobDesc *jobs = nullptr;
  TileDesc *tiles = nullptr;
  ClusterSlot *slots = nullptr;
  ApplyClusterSlot *aslots = nullptr;
  int32_t *err = nullptr;  // the device error word
  ~DevPlan() {
    int cur = 0;
    cudaGetDevice(&cur);
    if (device >= 0) cudaSetDevice(device);
    if (jobs) cudaFree(jobs);
    if (tiles) cudaFree(tiles);
    if (slots) cudaFree(slots);
    if (aslots) cudaFree(aslots);
    cudaSetDevice(cur);
  }
};

static std::mutex g_plan_mu;
static std::list<std::shared_ptr<DevPlan>> g_plans;  // most recent first
constexpr size_t kPlanCacheSize = 64;

static tsqr_status get_plan(int64_t m, int n, int nc, int leaf_h, int arity, int flags,
                            std::shared_ptr<DevPlan> &out) {
  const bool mixed = false;  // the mixed path plans through the batched engine
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  flags &= (TSQR_TWO_LEVEL | TSQR_CLUSTER);
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (auto it = g_plans.begin(); it != g_plans.end(); ++it) {
      const Plan &p = (*it)->plan;
      if ((*it)->device == dev && p.m == m && p.n == n && p.nc == nc && p.leaf_h == leaf_h &&
          p.arity == arity && p.flags == flags && p.mixed == mixed) {
        out = *it;
        g_plans.splice(g_plans.begin(), g_plans, it);
        return TSQR_OK;
      }
    }
  }
  const DeviceInfo di = device_info(dev);
  if (di.sms == 0) return fail(TSQR_ERR_CUDA, "cannot query device %d", dev);
  auto dp = std::make_shared<DevPlan>();
  dp->device = dev;
  tsqr_status st = make_plan_on(di, dp->plan, m, n, nc, leaf_h, arity, flags, mixed);
  if (st != TSQR_OK) return st;
  const Plan &pl = dp->plan;
  CUDA_TRY(cudaMalloc(&dp->jobs, sizeof(JobDesc) * pl.jobs.size()));
  CUDA_TRY(cudaMalloc(&dp->tiles, sizeof(TileDesc) * pl.tiles.size()));
  CUDA_TRY(cudaMemcpy(dp->jobs, pl.jobs.data(), sizeof(JobDesc) * pl.jobs.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(dp->tiles, pl.tiles.data(), sizeof(TileDesc) * pl.tiles.size(), cudaMemcpyHostToDevice));
  if (!pl.cl_slots.empty()) {
    CUDA_TRY(cudaMalloc(&dp->slots, sizeof(ClusterSlot) * pl.cl_slots.size()));
    CUDA_TRY(cudaMemcpy(dp->slots, pl.cl_slots.data(), sizeof(ClusterSlot) * pl.cl_slots.size(),
                        cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&dp->aslots, sizeof(ApplyClusterSlot) * pl.cl_apply.size()));
    CUDA_TRY(cudaMemcpy(dp->aslots, pl.cl_apply.data(), sizeof(ApplyClusterSlot) * pl.cl_apply.size(),
                        cudaMemcpyHostToDevice));
  }
  CUDA_TRY(device_error_word(&dp->err));
  std::lock_guard<std::mutex> lk(g_plan_mu);
  g_plans.push_front(dp);
  while (g_plans.size() > kPlanCacheSize) g_plans.pop_back();
  out = dp;
  return TSQR_OK;
}

struct tsqr_factors {
  std::shared_ptr<DevPlan> dp;
  int device = 0;
  cudaStream_t stream = nullptr;
  double *V = nullptr;  // reflector storage (== user A when in place)
  int64_t ldv = 0;
  bool owns_V = false;
  double *tau = nullptr, *scl = nullptr, *d = nullptr;
  void *block = nullptr;  // one allocation for tau, scl, d
  // CAQR (tsqr_caqr): the TSQR factor sets of the panels in order; panel p covers columns
  // p*panel.. and rows p*panel..m-1 of V, the m-by-ncols working copy that holds every
  // panel's reflectors. Rfull is the ncols-by-ncols R with diag >= 0.
  std::vector<tsqr_factors *> panels;
  int32_t panel = 0, ncols = 0;
  int64_t mrows = 0;
  double *Rfull = nullptr;
  bool caqr() const { return !panels.empty(); }
  const Plan &plan() const { return dp->plan; }
  int64_t rows() const { return caqr() ? mrows : dp->plan.m; }
  int32_t cols() const { return caqr() ? ncols : dp->plan.n; }
};

static tsqr_status factors_alloc(tsqr_factors *F, cudaStream_t s) {
  const Plan &pl = F->plan();
  const size_t nrefl = pl.tiles.size() * (size_t)pl.n;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_tau = up(sizeof(double) * nrefl), b_d = up(sizeof(double) * pl.n);
  CUDA_TRY(pool_alloc(&F->block, 2 * b_tau + b_d, s));
  char *base = (char *)F->block;
  F->tau = (double *)base;
  F->scl = (double *)(base + b_tau);
  F->d = (double *)(base + 2 * b_tau);
  return TSQR_OK;
}

static void factors_release(tsqr_factors *F) {
  if (!F) return;
  for (tsqr_factors *P : F->panels) factors_release(P);
  if (F->Rfull) cudaFreeAsync(F->Rfull, F->stream);
  if (F->block) cudaFreeAsync(F->block, F->stream);
  if (F->owns_V && F->V) cudaFreeAsync(F->V, F->stream);
  delete F;
}

// The bounds a TSQR_CHECK build checks every job and tile descriptor against.
template <typename P>
static void set_bounds(const tsqr_factors *F, P &p) {
  const Plan &pl = F->plan();
  p.rows = pl.m;
  p.nrefl = (int64_t)pl.tiles.size() * pl.n;
  p.ntiles = (int32_t)pl.tiles.size();
  p.njobs = (int32_t)pl.jobs.size();
  p.err = F->dp->err;
}

// Factorization launch q of F's plan: the chain launch (q = 0), then one tree level per
// launch, or with TSQR_CLUSTER one cluster launch per three levels. p.job0 is set here.
static cudaError_t factor_launch(const tsqr_factors *F, FactorParams &p, int q, cudaStream_t s) {
  const Plan &pl = F->plan();
  if (q > pl.cl_base && !pl.cl_launches.empty()) {
    const Plan::ClusterLaunch &cl = pl.cl_launches[q - 1 - pl.cl_base];
    p.job0 = 0;
    ProfScope ps(TSQR_PROF_FACTOR_TREE, s);
    return launch_factor_cluster(p, F->dp->slots + cl.slot_begin, cl.nclusters,
                                 F->dp->err, s);
  }
  const LaunchDesc &ld = pl.launches[q];
  p.job0 = ld.job_begin;
  ProfScope ps(q == 0 ? TSQR_PROF_FACTOR_CHAINS : TSQR_PROF_FACTOR_TREE, s);
  return launch_factor(p, ld.job_count, s, q == 0 ? pl.ctas_per_sm : 2);
}

// The binary tree levels (apply launches) that factorization launch q completes.
static void factor_launch_levels(const Plan &pl, int q, int &lo, int &hi) {
  if (q > pl.cl_base && !pl.cl_launches.empty()) {
    lo = pl.cl_launches[q - 1 - pl.cl_base].level_lo;
    hi = pl.cl_launches[q - 1 - pl.cl_base].level_hi;
  } else {
    lo = hi = q;
  }
}

// Runs the factorization launches of F on A (first touch) and optional extra columns B.
static tsqr_status run_factor(tsqr_factors *F, const double *A, int64_t lda, double *B, int64_t ldb,
                              cudaStream_t s) {
  const Plan &pl = F->plan();
  FactorParams p{};
  p.A = A;
  p.lda = lda;
  p.V = F->V;
  p.ldv = F->ldv;
  p.B = B;
  p.ldb = ldb;
  p.jobs = F->dp->jobs;
  p.tiles = F->dp->tiles;
  p.tau = F->tau;
  p.scl = F->scl;
  p.n = pl.n;
  p.nc = B ? pl.nc : pl.n;
  p.ldt = pl.tile_h;
  set_bounds(F, p);
  for (int q = 0; q < pl.factor_launches(); ++q) CUDA_TRY(factor_launch(F, p, q, s));
  return TSQR_OK;
}

// Launch li of the plan applied to B's columns [c0, c0 + kg) (kg <= 64; the warp kernel
// for kg <= 8): Q^T in forward launch order, Q in reverse.
static tsqr_status apply_launch(const tsqr_factors *F, double *B, int64_t ldb, int c0, int kg, int trans, int formq,
                                int li, cudaStream_t s) {
  const Plan &pl = F->plan();
  ApplyParams p{};
  p.V = F->V;
  p.ldv = F->ldv;
  p.B = B;
  p.ldb = ldb;
  p.jobs = F->dp->jobs;
  p.tiles = F->dp->tiles;
  p.tau = F->tau;
  p.scl = F->scl;
  p.n = pl.n;
  p.ldt = pl.tile_h;
  p.trans = trans;
  p.formq = formq;
  p.col0 = c0;
  p.k = kg;
  set_bounds(F, p);
  const LaunchDesc &ld = pl.launches[li];
  p.job0 = ld.job_begin;
  const int sms = device_info(F->device).sms;
  ProfScope ps(formq ? TSQR_PROF_FORM_Q : (trans ? TSQR_PROF_APPLY_QT : TSQR_PROF_APPLY_Q), s);
  // a tree level whose nodes, four CTAs each, still fit one wave of two CTAs per SM runs
  // 16 columns per CTA: each node's reflector steps get shorter
  const bool narrow = li > 0 && (int64_t)ld.job_count * 4 <= (int64_t)sms * 2;
  // one column over jobs of several tiles (the chains): tile pairs per warp
  const bool pairs = ld.job_count > 0 && pl.jobs[ld.job_begin].tile_count >= 2 && g_tile_pairs.load() != 0;
  CUDA_TRY(launch_apply(p, ld.job_count, s, li == 0 ? pl.ctas_per_sm : 2, narrow ? 16 : 64, pairs));
  return TSQR_OK;
}

// B is processed in groups of at most 64 columns (8 for the warp kernel path)
static int apply_group(int k) { return (k <= 8) ? 8 : 64; }

// The thin Q of up to 32 columns is formed in passes of 4 columns by the warp kernel: at
// these widths the CTA kernel leaves most of its half-warps idle (reflector j touches
// columns >= j only) between block barriers, and 4 columns per warp keep a job's staged
// tile small enough for two or three CTAs of four jobs per SM.
static int formq_group(int n) { return (n <= 32) ? 4 : 64; }

// The cluster launch of F's plan that completes tree level li top down (the launch whose
// highest level is li), for the columns [c0, c0 + kg) of B.
static tsqr_status apply_cluster_launch(const tsqr_factors *F, double *B, int64_t ldb, int c0, int kg, int formq,
                                        const Plan::ClusterLaunch &cl, cudaStream_t s) {
  const Plan &pl = F->plan();
  ApplyParams p{};
  p.V = F->V;
  p.ldv = F->ldv;
  p.B = B;
  p.ldb = ldb;
  p.jobs = F->dp->jobs;
  p.tiles = F->dp->tiles;
  p.tau = F->tau;
  p.scl = F->scl;
  p.n = pl.n;
  p.ldt = pl.n;
  p.trans = 0;
  p.formq = formq;
  p.col0 = c0;
  p.k = kg;
  set_bounds(F, p);
  ProfScope ps(formq ? TSQR_PROF_FORM_Q : TSQR_PROF_APPLY_Q, s);
  CUDA_TRY(launch_apply_cluster(p, F->dp->aslots + cl.slot_begin, cl.nclusters, s));
  return TSQR_OK;
}

static tsqr_status run_apply(const tsqr_factors *F, double *B, int64_t ldb, int k, int trans, int formq,
                             cudaStream_t s) {
  const Plan &pl = F->plan();
  const int nl = (int)pl.launches.size();
  const int group = formq ? formq_group(k) : apply_group(k);
  // Q B top down with groups of more than 8 columns (the tile kernel's arithmetic, which the
  // cluster launches share, so results stay bitwise those of the per-level launches): the
  // levels of the cluster launches run as cluster launches, highest first
  for (int c0 = 0; c0 < k; c0 += group) {
    const int kg = std::min(group, k - c0);
    const bool clustered = !trans && kg > 8 && !pl.cl_launches.empty() && F->dp->aslots;
    for (int q = 0; q < nl; ++q) {
      const int li = trans ? q : nl - 1 - q;
      tsqr_status st = TSQR_OK;
      // a cluster launch runs only while all its CTAs (16 columns each) fit one wave at two
      // per SM: on wider levels the pipelined launch is slower than the per-level launches
      // (measured at 4M x 64: levels 3-5 of the thin Q 0.65 ms clustered, 0.43 ms per level)
      const Plan::ClusterLaunch *hit = nullptr;
      if (clustered && li > pl.cl_base)
        for (const Plan::ClusterLaunch &cl : pl.cl_launches)
          if (li >= cl.level_lo && li <= cl.level_hi) hit = &cl;
      const int sms = device_info(F->device).sms;
      if (hit && (int64_t)hit->nclusters * kClusterSize * ((kg + 15) / 16) > (int64_t)sms * 2) hit = nullptr;
      if (hit) {
        if (li == hit->level_hi) st = apply_cluster_launch(F, B, ldb, c0, kg, formq, *hit, s);
      } else {
        st = apply_launch(F, B, ldb, c0, kg, trans, formq, li, s);
      }
      if (st != TSQR_OK) return st;
    }
  }
  return TSQR_OK;
}

static tsqr_status check_factor_args(const void *A, int64_t m, int32_t n, int64_t lda, int32_t leaf_h,
                                     int32_t arity) {
  if (!A) return fail(TSQR_ERR_ARG, "A is NULL");
  if (n < 1 || n > 128) return fail(TSQR_ERR_ARG, "n=%d outside [1, 128] (tsqr_caqr factors wider matrices)", n);
  if (m < n) return fail(TSQR_ERR_ARG, "m=%lld < n=%d", (long long)m, n);
  if (lda < m) return fail(TSQR_ERR_ARG, "lda=%lld < m=%lld", (long long)lda, (long long)m);
  if (leaf_h < n) return fail(TSQR_ERR_ARG, "leaf_h=%d < n=%d", leaf_h, n);
  if (!(arity == 0 || (arity >= 2 && arity <= 16))) return fail(TSQR_ERR_ARG, "arity=%d not in {0, 2..16}", arity);
  return TSQR_OK;
}

static void plan_info(const Plan &pl, int64_t *out) {
  out[0] = pl.m;
  out[1] = pl.n;
  out[2] = pl.leaves;
  out[3] = pl.tile_h;
  out[4] = (int64_t)pl.jobs.size();
  out[5] = (int64_t)pl.tiles.size();
  out[6] = (int64_t)pl.factor_launches() + 1;
  out[7] = pl.ctas_per_sm;
}

// Batched mixed least squares (refine_batch.cu): rows per refinement task, the number of
// refinement launches, and the stopping tolerance on the predicted remaining
// ||dX||/||X|| (the last correction times rho / (1 - rho), rho the observed contraction).
// the batched autotuner's candidates (tsqr_batch_autotune's ms_table order: chain tiles
// outer, arity inner)
constexpr int32_t kBatchTuneChainTiles[] = {2, 4, 8, 16, 32};
constexpr int32_t kBatchTuneArity[] = {2, 4};
constexpr int64_t kRefineRows = 4096;
constexpr size_t kBatchSmemSlack = 256;
constexpr int kMixedChainFactor = 4;
constexpr int32_t kRefineSteps = 10;
// the refinement stops once its predicted remaining ||dX|| / ||X|| is below this: the
// accuracy the mixed path is held to (1e-10 from the FP64 solution for kappa <= 1e4). The
// prediction (last correction x rho / (1 - rho), rho the largest ratio of successive
// corrections) overestimates: over 200 served-mix and kappa = 1e4, noise 1e-3 problems the
// error at the stop was at most 9.7e-12 (at most 4.2e-13 with 1e-12, 11% more steps).
constexpr double kBatchRefineTol = 1e-10;
// Cost model of TSQR_AUTO, in TFLOP/s as the kernels run inside a GB300 batch of served
// requests: the FP64 factor kernel (lower for n < 32, where the column steps are short),
// the FP32 register-tile factor kernel (rising with n up to its plateau), the refinement
// kernel, and the refinement steps counted at full cost (the first step, from x = 0,
// costs half). Fitted so that, in a served mix, only n = 16 requests with k >= 6 take
// FP64 (timing every policy over the same 128 requests: the others were slower).
constexpr double kFp64Factor = 0.76, kFp64FactorNarrow = 0.5;
constexpr double kFp32FactorPerCol = 0.1, kFp32FactorMax = 6.0;
constexpr double kRefineTflops = 0.75, kRefineTflopsNarrow = 0.6;
constexpr double kRefineStepsEst = 2.3;

// ---------------------------------------------------------------- batched solve
namespace {

// Everything the batched path plans on the host for one set of items: the per-item
// plans, the merged job and tile tables, the refinement tables, and the layout of the
// one device block that holds workspaces and tables.
struct BatchBuild {
  int32_t count = 0;
  std::vector<tsqr_batch_item> items;
  std::vector<Plan> plans;
  std::vector<int32_t> prec, tree_rows, wy;
  bool wy_any = false;
  size_t smem = 0;
  int cmax = 1, grid = 0;
  int32_t nchains = 0, njobs = 0;
  int64_t ntiles = 0;
  std::vector<BatchJob> jobs;
  std::vector<TileDesc> tiles;
  std::vector<int64_t> root;  // where each item's R lands in its tree storage
  struct Off {
    size_t V, B, tau, scl, V64, tau64, scl64;
  };
  std::vector<Off> offs;
  size_t o_inst = 0, o_jobs = 0, o_tiles = 0, o_cnt = 0, o_st = 0;
  size_t o_rinst = 0, o_rtasks = 0, o_rflags = 0, o_rhist = 0, bytes = 0;
  std::vector<int32_t> ritem;  // item of each refinement instance
  std::vector<size_t> rP;      // its partials
  std::vector<BatchInst> inst;
  std::vector<RefineInst> rinst;
  std::vector<RefineTask> rtasks;
  size_t rsmem = 0;
  int32_t max_steps = kRefineSteps;  // refinement launches (mixed least-squares items)
};

tsqr_status batch_build_on(DeviceInfo di, const tsqr_batch_item *items, int32_t count, int32_t chain_tiles,
                           int32_t arity, BatchBuild &b, int32_t max_steps, int32_t ctas_per_sm);

tsqr_status batch_build(const tsqr_batch_item *items, int32_t count, int32_t chain_tiles, int32_t arity,
                        BatchBuild &b, int32_t max_steps = kRefineSteps, int32_t ctas_per_sm = 0) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  const DeviceInfo di = device_info(dev);
  if (di.sms == 0) return fail(TSQR_ERR_CUDA, "cannot query device %d", dev);
  return batch_build_on(di, items, count, chain_tiles, arity, b, max_steps, ctas_per_sm);
}

// The host planning of a batch for a device described by di (no CUDA call).
tsqr_status batch_build_on(DeviceInfo di, const tsqr_batch_item *items, int32_t count, int32_t chain_tiles,
                           int32_t arity, BatchBuild &b, int32_t max_steps, int32_t ctas_per_sm) {
  b.max_steps = max_steps;
  // the persistent kernel has a few bytes of static shared memory, and allocations are
  // rounded up: budget for both so that two CTAs per SM still fit where planned
  di.reserved += kBatchSmemSlack;
  if (arity == 0) arity = 2;
  const int L = chain_tiles > 0 ? chain_tiles : 8;
  b.count = count;
  b.items.assign(items, items + count);
  b.plans.resize(count);
  b.prec.resize(count);
  b.tree_rows.resize(count);
  b.wy.assign(count, 0);
  const int32_t wy_min = g_wy_min_n.load();
  int cps_min = 2;
  bool any_refine = false;
  for (int32_t q = 0; q < count; ++q) {
    const tsqr_batch_item &it = items[q];
    b.prec[q] = resolve_batch_prec(it);
    const bool mixed = b.prec[q] == TSQR_MIXED;
    any_refine = any_refine || (mixed && it.k > 0);
    // FP64 items fuse Q^T B into the factorization; mixed items factor A alone and
    // solve by refinement afterwards
    const int nc = mixed ? it.n : it.n + it.k;
    const size_t elem = mixed ? sizeof(float) : sizeof(double);
    int th = 0, cps = 0;
    if (!choose_tiles(di, it.n, nc, 1 << 20, th, cps, elem, 2))
      return fail(TSQR_ERR_UNSUPPORTED, "item %d: no tile fits shared memory", q);
    const int64_t tiles = (it.m + th - 1) / th;
    // mixed items: FP32 chains kMixedChainFactor times longer (fewer FP64 tree combines)
    const int64_t Lq = mixed ? (int64_t)L * kMixedChainFactor : L;
    const int64_t G = std::max<int64_t>(1, (tiles + Lq / 2) / Lq);
    tsqr_status st = make_plan_on(di, b.plans[q], it.m, it.n, nc, th, arity, TSQR_TWO_LEVEL, mixed, G, 2);
    if (st != TSQR_OK) return st;
    // tree nodes (FP64) in pieces that fit the chains' CTAs per SM
    const int node_rows = b.tree_rows[q] = split_tree_tiles(
        b.plans[q], factor_max_rows(nc, b.plans[q].ctas_per_sm, di.smem_sm, di.reserved, di.optin, sizeof(double)));
    size_t chain_smem = factor_smem_bytes(nc, b.plans[q].tile_h, elem);
    if (mixed && wy_min > 0 && it.n >= wy_min && it.n > 16) {
      // compact-WY FP32 chains, if their buffers still fit two CTAs per SM
      const size_t wsm = chain_smem + f32wy_smem_extra_bytes();
      if (wsm <= di.optin && 2 * (wsm + di.reserved) <= di.smem_sm) {
        chain_smem = wsm;
        b.wy[q] = 1;
        b.wy_any = true;
      }
    }
    b.smem = std::max(b.smem, chain_smem);
    b.smem = std::max(b.smem, factor_smem_bytes(nc, node_rows, sizeof(double)));
    b.smem = std::max(b.smem, sizeof(double) * (size_t)it.n * std::max(it.k, 1));
    while (16 * b.cmax < nc) b.cmax *= 2;
    cps_min = std::min(cps_min, b.plans[q].ctas_per_sm);
  }
  // ctas_per_sm = 1 leaves room on every SM for a CTA of another stream's kernel (the
  // server overlaps one batch's refinement with the next batch's factorization)
  b.grid = di.sms * (ctas_per_sm > 0 ? std::min(cps_min, (int)ctas_per_sm) : cps_min);
  // merged job table: chains of every item (largest first), then tree nodes
  struct Chain {
    double cost;
    int32_t item, job;
  };
  std::vector<Chain> chains;
  std::vector<int64_t> tile_base(count);
  for (int32_t q = 0; q < count; ++q) {
    const Plan &pl = b.plans[q];
    tile_base[q] = b.ntiles;
    b.ntiles += (int64_t)pl.tiles.size();
    for (int32_t c = 0; c < pl.launches[0].job_count; ++c) {
      const JobDesc &jd = pl.jobs[c];
      double rows = 0;
      for (int32_t t = jd.tile_begin; t < jd.tile_begin + jd.tile_count; ++t) rows += pl.tiles[t].nrows;
      const double w = (double)(pl.nc) * pl.nc * (pl.mixed ? 0.1 : 1.0);
      chains.push_back({rows * w, q, c});
    }
  }
  std::sort(chains.begin(), chains.end(), [](const Chain &x, const Chain &y) { return x.cost > y.cost; });
  b.nchains = (int32_t)chains.size();
  std::vector<std::vector<int32_t>> gidx(count);  // global job index of each plan job
  for (int32_t q = 0; q < count; ++q) gidx[q].assign(b.plans[q].jobs.size(), -1);
  for (int32_t c = 0; c < b.nchains; ++c) gidx[chains[c].item][chains[c].job] = c;
  int32_t next = b.nchains;
  for (int32_t q = 0; q < count; ++q)
    for (size_t j = b.plans[q].launches[0].job_count; j < b.plans[q].jobs.size(); ++j) gidx[q][j] = next++;
  b.njobs = next;
  b.jobs.resize(b.njobs);
  b.tiles.resize((size_t)b.ntiles);
  for (int32_t q = 0; q < count; ++q) {
    const Plan &pl = b.plans[q];
    std::copy(pl.tiles.begin(), pl.tiles.end(), b.tiles.begin() + tile_base[q]);
    const int32_t G = pl.launches[0].job_count;
    // parents: follow which job currently holds each pivot block, level by level
    std::vector<int32_t> holder(G);  // by chain index
    std::vector<std::pair<int64_t, int32_t>> rowkey(G);  // (tree-storage row, chain index)
    for (int32_t c = 0; c < G; ++c) {
      holder[c] = c;
      rowkey[c] = {pl.mixed ? (int64_t)c * pl.n : pl.jobs[c].piv_row, c};
    }
    std::sort(rowkey.begin(), rowkey.end());
    auto chain_of = [&](int64_t row) {
      return std::lower_bound(rowkey.begin(), rowkey.end(), std::make_pair(row, (int32_t)-1))->second;
    };
    for (int32_t c = 0; c < G; ++c) {
      BatchJob &bj = b.jobs[gidx[q][c]];
      const JobDesc &jd = pl.jobs[c];
      bj.piv_row = jd.piv_row;
      bj.row64 = pl.mixed ? (int64_t)c * pl.n : jd.piv_row;
      bj.tile_begin = (int32_t)(tile_base[q] + jd.tile_begin);
      bj.tile_count = jd.tile_count;
      bj.inst = q;
      bj.parent = -1;
      bj.nchild = 0;
    }
    for (size_t j = G; j < pl.jobs.size(); ++j) {
      const JobDesc &jd = pl.jobs[j];
      BatchJob &bj = b.jobs[gidx[q][j]];
      bj.piv_row = jd.piv_row;
      bj.row64 = jd.piv_row;
      bj.tile_begin = (int32_t)(tile_base[q] + jd.tile_begin);
      bj.tile_count = jd.tile_count;
      bj.inst = q;
      bj.parent = -1;
      int32_t nchild = 1;
      const int32_t first = chain_of(jd.piv_row);
      b.jobs[gidx[q][holder[first]]].parent = gidx[q][j];
      for (int32_t t = jd.tile_begin; t < jd.tile_begin + jd.tile_count; ++t) {
        if (pl.tiles[t].off != 0) continue;  // a later piece of the same child
        b.jobs[gidx[q][holder[chain_of(pl.tiles[t].row0)]]].parent = gidx[q][j];
        ++nchild;
      }
      bj.nchild = nchild;
      holder[first] = (int32_t)j;
    }
  }
  b.root.assign(count, -1);
  for (int32_t j = 0; j < b.njobs; ++j)
    if (b.jobs[j].parent < 0) b.root[b.jobs[j].inst] = b.jobs[j].row64;
  // device block: per-item workspaces, then the tables
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t off = 0;
  auto take = [&](size_t x) {
    const size_t o = off;
    off += up(x);
    return o;
  };
  b.offs.resize(count);
  for (int32_t q = 0; q < count; ++q) {
    const tsqr_batch_item &it = items[q];
    const Plan &pl = b.plans[q];
    const size_t elem = pl.mixed ? sizeof(float) : sizeof(double);
    const size_t nrefl = pl.tiles.size() * (size_t)it.n;
    BatchBuild::Off &o = b.offs[q];
    o = {};
    o.V = take(elem * (size_t)it.m * it.n);
    o.B = (!pl.mixed && it.k > 0) ? take(sizeof(double) * (size_t)it.m * it.k) : 0;
    o.tau = take(elem * nrefl);
    o.scl = take(elem * nrefl);
    if (pl.mixed) {
      const int64_t Gn = (int64_t)pl.launches[0].job_count * it.n;
      o.V64 = take(sizeof(double) * (size_t)Gn * it.n);
      o.tau64 = take(sizeof(double) * nrefl);
      o.scl64 = take(sizeof(double) * nrefl);
    }
  }
  b.o_inst = take(sizeof(BatchInst) * count);
  b.o_jobs = take(sizeof(BatchJob) * b.njobs);
  b.o_tiles = take(sizeof(TileDesc) * (size_t)b.ntiles);
  b.o_cnt = take(sizeof(int32_t) * ((size_t)b.njobs + 1));
  b.o_st = take(sizeof(int32_t) * count);
  // refinement of mixed least-squares items: one instance per group of <= 8 right-hand
  // sides, tasks of kRefineRows rows
  for (int32_t q = 0; q < count && any_refine; ++q) {
    const tsqr_batch_item &it = items[q];
    if (b.prec[q] != TSQR_MIXED || it.k == 0) continue;
    if (b.root[q] < 0) return fail(TSQR_ERR_CUDA, "item %d: the plan has no root job", q);
    const int32_t nt = (int32_t)((it.m + kRefineRows - 1) / kRefineRows);
    for (int32_t c0 = 0; c0 < it.k; c0 += 8) {
      RefineInst ri{};
      ri.n = it.n;
      ri.k = std::min(8, it.k - c0);
      ri.kb = ri.k;
      ri.nt = nt;
      ri.A = it.A;
      ri.lda = it.lda;
      ri.B = it.B + (int64_t)c0 * it.ldb;
      ri.ldb = it.ldb;
      ri.X = it.X + (int64_t)c0 * it.ldx;
      ri.ldx = it.ldx;
      ri.ldr = (int64_t)b.plans[q].launches[0].job_count * it.n;  // compact FP64 tree storage
      const int32_t ix = (int32_t)b.rinst.size();
      for (int32_t t = 0; t < nt; ++t) {
        RefineTask tk{};
        tk.row0 = (int64_t)t * kRefineRows;
        tk.rows = (int32_t)std::min<int64_t>(kRefineRows, it.m - tk.row0);
        tk.inst = ix;
        tk.idx = t;
        b.rtasks.push_back(tk);
      }
      b.rP.push_back(take(sizeof(double) * (size_t)nt * it.n * ri.k));
      b.ritem.push_back(q);
      b.rinst.push_back(ri);
      b.rsmem = std::max(b.rsmem, refine_smem_bytes(it.n, ri.kb));
    }
  }
  if (!b.rinst.empty()) {
    b.o_rhist = take(sizeof(double) * b.max_steps * b.rinst.size());
    b.o_rinst = take(sizeof(RefineInst) * b.rinst.size());
    b.o_rtasks = take(sizeof(RefineTask) * b.rtasks.size());
    b.o_rflags = take(sizeof(int32_t) * 2 * b.rinst.size());
  }
  b.bytes = off;
  return TSQR_OK;
}

// Fills the device addresses of the instance and refinement tables for a block at base.
void batch_bind(BatchBuild &b, char *base) {
  b.inst.resize(b.count);
  for (int32_t q = 0; q < b.count; ++q) {
    const tsqr_batch_item &it = b.items[q];
    const Plan &pl = b.plans[q];
    const BatchBuild::Off &o = b.offs[q];
    BatchInst &bi = b.inst[q];
    bi = {};
    bi.A = it.A;
    bi.lda = it.lda;
    bi.V = base + o.V;
    bi.ldv = it.m;
    bi.ldb = it.m;
    bi.tau = base + o.tau;
    bi.scl = base + o.scl;
    if (pl.mixed) {
      bi.V64 = (double *)(base + o.V64);
      bi.ldv64 = (int64_t)pl.launches[0].job_count * it.n;
      bi.tau64 = (double *)(base + o.tau64);
      bi.scl64 = (double *)(base + o.scl64);
    } else {
      bi.V64 = (double *)bi.V;
      bi.ldv64 = it.m;
      bi.tau64 = (double *)bi.tau;
      bi.scl64 = (double *)bi.scl;
    }
    bi.R = it.R;
    bi.ldr = it.ldr;
    bi.X = pl.mixed ? nullptr : it.X;  // mixed items are solved by the refinement launches
    bi.ldx = it.ldx;
    bi.status = (int32_t *)(base + b.o_st) + q;
    bi.n = it.n;
    bi.k = pl.mixed ? 0 : it.k;
    bi.B = bi.k > 0 ? (double *)(base + o.B) : nullptr;
    bi.ldt = pl.tile_h;
    bi.ldt_tree = b.tree_rows[q];
    bi.mixed = pl.mixed ? 1 : 0;
    bi.wy = b.wy[q];
  }
  int32_t *flags = (int32_t *)(base + b.o_rflags);  // counter, done per instance
  for (size_t r = 0; r < b.rinst.size(); ++r) {
    const int32_t q = b.ritem[r];
    RefineInst &ri = b.rinst[r];
    ri.R = b.inst[q].V64 + b.root[q];
    ri.P = (double *)(base + b.rP[r]);
    ri.hist = (double *)(base + b.o_rhist) + (size_t)b.max_steps * r;
    ri.counter = flags + 2 * r;
    ri.done = flags + 2 * r + 1;
    ri.status = (int32_t *)(base + b.o_st) + q;
  }
}

// The tables, host to device. A copy from pageable memory may wait for the stream to
// drain, so this is issued before any kernel of the call.
tsqr_status batch_upload(const BatchBuild &b, char *base, cudaStream_t s) {
  CUDA_TRY(cudaMemcpyAsync(base + b.o_inst, b.inst.data(), sizeof(BatchInst) * b.count, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(base + b.o_jobs, b.jobs.data(), sizeof(BatchJob) * b.njobs, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(base + b.o_tiles, b.tiles.data(), sizeof(TileDesc) * (size_t)b.ntiles,
                           cudaMemcpyHostToDevice, s));
  if (!b.rinst.empty()) {
    CUDA_TRY(cudaMemcpyAsync(base + b.o_rinst, b.rinst.data(), sizeof(RefineInst) * b.rinst.size(),
                             cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(base + b.o_rtasks, b.rtasks.data(), sizeof(RefineTask) * b.rtasks.size(),
                             cudaMemcpyHostToDevice, s));
  }
  return TSQR_OK;
}

// One run: the right-hand-side copies, counter and flag resets, the persistent kernel,
// and the refinement launches. Device-side operations only, so it can be captured in a
// CUDA graph.
tsqr_status batch_enqueue(const BatchBuild &b, char *base, cudaStream_t s, bool profile) {
  for (int32_t q = 0; q < b.count; ++q) {
    const tsqr_batch_item &it = b.items[q];
    const BatchInst &bi = b.inst[q];
    if (bi.k > 0)
      CUDA_TRY(cudaMemcpy2DAsync(bi.B, sizeof(double) * it.m, it.B, sizeof(double) * it.ldb, sizeof(double) * it.m,
                                 it.k, cudaMemcpyDeviceToDevice, s));
  }
  CUDA_TRY(cudaMemsetAsync(base + b.o_cnt, 0, sizeof(int32_t) * ((size_t)b.njobs + 1), s));
  CUDA_TRY(cudaMemsetAsync(base + b.o_st, 0, sizeof(int32_t) * b.count, s));
  if (!b.rinst.empty()) {
    CUDA_TRY(cudaMemsetAsync(base + b.o_rflags, 0, sizeof(int32_t) * 2 * b.rinst.size(), s));
    // all-ones bytes are a NaN: "step not run" for the history readback
    CUDA_TRY(cudaMemsetAsync(base + b.o_rhist, 0xff, sizeof(double) * b.max_steps * b.rinst.size(), s));
  }
  BatchParams bp{};
  bp.inst = (const BatchInst *)(base + b.o_inst);
  bp.jobs = (const BatchJob *)(base + b.o_jobs);
  bp.tiles = (const TileDesc *)(base + b.o_tiles);
  bp.counters = (int32_t *)(base + b.o_cnt);
  bp.queue = bp.counters + b.njobs;
  bp.nchains = b.nchains;
  {
    ProfScope ps(profile ? TSQR_PROF_BATCH : -1, s);
    CUDA_TRY(launch_factor_batch(bp, b.cmax, b.grid, b.smem, s, b.wy_any));
  }
  if (!b.rinst.empty()) {
    RefineParams rp{};
    rp.inst = (const RefineInst *)(base + b.o_rinst);
    rp.tasks = (const RefineTask *)(base + b.o_rtasks);
    rp.max_steps = b.max_steps;
    rp.tol = kBatchRefineTol;
    ProfScope ps(profile ? TSQR_PROF_REFINE : -1, s);
    for (int32_t step = 0; step < b.max_steps; ++step) {
      rp.step = step;
      CUDA_TRY(launch_refine_batch(rp, (int)b.rtasks.size(), b.rsmem, s));
    }
  }
  return TSQR_OK;
}

// Per-item (steps run, last ||dX||/||X||) from a host copy of the refinement history.
void batch_info(const BatchBuild &b, const double *hist, double *info) {
  for (int32_t q = 0; q < b.count; ++q) info[2 * q] = info[2 * q + 1] = 0.0;
  for (size_t r = 0; r < b.rinst.size(); ++r) {
    int steps = 0;
    while (steps < b.max_steps && hist[(size_t)b.max_steps * r + steps] >= 0.0) ++steps;
    double *o = info + 2 * b.ritem[r];
    o[0] = std::max(o[0], (double)steps);
    if (steps > 0) o[1] = std::max(o[1], hist[(size_t)b.max_steps * r + steps - 1]);
  }
}

// One mixed least-squares problem through the batched engine: FP32 chains, FP64 tree,
// corrected semi-normal-equation refinement, at most max_steps steps. hist (host,
// max_steps doubles, or NULL) receives ||dX||/||X|| per step, the largest over the groups
// of 8 right-hand sides (0 for steps not run).
tsqr_status lstsq_mixed_batched(const tsqr_batch_item &it, int32_t arity, int32_t max_steps, cudaStream_t s,
                                double *hist) {
  BatchBuild b;
  tsqr_status st = batch_build(&it, 1, 0, arity, b, max_steps);
  if (st != TSQR_OK) return st;
  void *blk = nullptr;
  CUDA_TRY(pool_alloc(&blk, b.bytes, s));
  char *base = (char *)blk;
  batch_bind(b, base);
  st = batch_upload(b, base, s);
  if (st == TSQR_OK) st = batch_enqueue(b, base, s, true);
  int32_t hstatus = 0;
  std::vector<double> h((size_t)b.max_steps * b.rinst.size());
  if (st == TSQR_OK) {
    cudaError_t e = cudaMemcpyAsync(&hstatus, base + b.o_st, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && hist)
      e = cudaMemcpyAsync(h.data(), base + b.o_rhist, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "status readback: %s", cudaGetErrorString(e));
  }
  cudaFreeAsync(blk, s);
  if (st != TSQR_OK) return st;
  if (hist) {
    for (int32_t step = 0; step < b.max_steps; ++step) {
      double v = 0.0;
      for (size_t r = 0; r < b.rinst.size(); ++r) {
        const double x = h[(size_t)b.max_steps * r + step];
        if (x >= 0.0) v = std::max(v, x);
      }
      hist[step] = v;
    }
  }
  if (hstatus == TSQR_ERR_SINGULAR) return fail(TSQR_ERR_SINGULAR, "R has a zero diagonal entry");
  return TSQR_OK;
}

}  // namespace

tsqr_status tsqr::batch_solve_internal(const tsqr_batch_item *items, int32_t count, int32_t chain_tiles,
                                       int32_t arity, cudaStream_t s, int32_t *status, int32_t *status_async,
                                       double *info, int32_t ctas_per_sm) {
  BatchBuild b;
  tsqr_status st = batch_build(items, count, chain_tiles, arity, b, kRefineSteps, ctas_per_sm);
  if (st != TSQR_OK) return st;
  void *blk = nullptr;
  CUDA_TRY(pool_alloc(&blk, b.bytes, s));
  char *base = (char *)blk;
  batch_bind(b, base);
  st = batch_upload(b, base, s);
  if (st == TSQR_OK) st = batch_enqueue(b, base, s, true);
  if (st != TSQR_OK) {
    cudaFreeAsync(blk, s);
    return st;
  }
  if (status_async) {
    cudaError_t e = cudaMemcpyAsync(status_async, base + b.o_st, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "status copy: %s", cudaGetErrorString(e));
  }
  if (status) {
    cudaError_t e = cudaMemcpyAsync(status, base + b.o_st, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "status readback: %s", cudaGetErrorString(e));
  }
  if (info) {
    std::vector<double> hist((size_t)b.max_steps * b.rinst.size());
    cudaError_t e = cudaSuccess;
    if (!hist.empty()) {
      e = cudaMemcpyAsync(hist.data(), base + b.o_rhist, sizeof(double) * hist.size(), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess)
      st = fail(TSQR_ERR_CUDA, "refinement history readback: %s", cudaGetErrorString(e));
    else
      batch_info(b, hist.data(), info);
  }
  cudaFreeAsync(blk, s);
  return st;
}

// ------------------------------------------------- requests of the resident kernel
// A request is planned exactly as a one-item batch (so it is bitwise the same request as
// tsqr_batch_solve solves alone) and laid out in one device block of the resident
// server's arena: the batched layout, then the count of refinement groups still running.
size_t tsqr::resident_smem_bytes(int ctas_per_sm) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  const DeviceInfo di = device_info(dev);
  if (di.sms == 0 || ctas_per_sm < 1) return 0;
  const size_t per = di.smem_sm / (size_t)ctas_per_sm;
  const size_t fixed = di.reserved + kBatchSmemSlack;
  if (per <= fixed) return 0;
  return std::min(per - fixed, di.optin);
}

int64_t tsqr::refine_rows_per_task() { return kRefineRows; }
int32_t tsqr::refine_max_steps() { return kRefineSteps; }
double tsqr::refine_tolerance() { return kBatchRefineTol; }

tsqr_status tsqr::resident_plan(const tsqr_batch_item &it, int32_t chain_tiles, ResidentPlan &out) {
  out = ResidentPlan{};
  tsqr_status st = check_batch_item(it, 0);
  if (st != TSQR_OK) return st;
  BatchBuild *b = new (std::nothrow) BatchBuild();
  if (!b) return fail(TSQR_ERR_OOM, "host memory for a plan");
  st = batch_build(&it, 1, chain_tiles, 2, *b);
  if (st != TSQR_OK) {
    delete b;
    return st;
  }
  out.impl = b;
  out.bytes = b->bytes + 256;  // + the refinement groups still running
  // the resident kernel runs the register-tile FP32 leaf; a compact-WY plan only asked
  // for more shared memory
  size_t smem = 0;
  for (int32_t q = 0; q < b->count; ++q) {
    const int nc = b->plans[q].mixed ? it.n : it.n + it.k;
    const size_t elem = b->plans[q].mixed ? sizeof(float) : sizeof(double);
    smem = std::max(smem, factor_smem_bytes(nc, b->plans[q].tile_h, elem));
    smem = std::max(smem, factor_smem_bytes(nc, b->tree_rows[q], sizeof(double)));
    smem = std::max(smem, sizeof(double) * (size_t)it.n * std::max(it.k, 1));
  }
  out.smem = std::max(smem, b->rsmem);
  out.cmax = b->cmax;
  out.nchains = b->nchains;
  out.njobs = b->njobs;
  out.ngroups = (int32_t)b->rinst.size();
  out.nt = b->rinst.empty() ? 0 : b->rinst[0].nt;
  out.wy = b->wy_any;
  return TSQR_OK;
}

void tsqr::resident_plan_free(ResidentPlan &p) {
  delete static_cast<BatchBuild *>(p.impl);
  p.impl = nullptr;
}

tsqr_status tsqr::resident_upload(const ResidentPlan &p, char *base, cudaStream_t s, ResItemDev &dev) {
  BatchBuild &b = *static_cast<BatchBuild *>(p.impl);
  batch_bind(b, base);
  tsqr_status st = batch_upload(b, base, s);
  if (st != TSQR_OK) return st;
  const tsqr_batch_item &it = b.items[0];
  const BatchInst &bi = b.inst[0];
  if (bi.k > 0)
    CUDA_TRY(cudaMemcpy2DAsync(bi.B, sizeof(double) * it.m, it.B, sizeof(double) * it.ldb, sizeof(double) * it.m,
                               it.k, cudaMemcpyDeviceToDevice, s));
  // counters, status and flags are cleared by copies (copy engines), never by kernels: the
  // resident kernel may hold every SM while these run
  int32_t *pending = (int32_t *)(base + b.bytes);
  const int32_t groups = (int32_t)b.rinst.size();
  const size_t n_cnt = sizeof(int32_t) * ((size_t)b.njobs + 1), n_st = sizeof(int32_t) * b.count;
  const size_t n_fl = sizeof(int32_t) * 2 * b.rinst.size(), n_hist = sizeof(double) * b.max_steps * b.rinst.size();
  std::vector<unsigned char> zeros(std::max({n_cnt, n_st, n_fl}), 0), ones(n_hist, 0xff);
  CUDA_TRY(cudaMemcpyAsync(base + b.o_cnt, zeros.data(), n_cnt, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(base + b.o_st, zeros.data(), n_st, cudaMemcpyHostToDevice, s));
  if (groups > 0) {
    CUDA_TRY(cudaMemcpyAsync(base + b.o_rflags, zeros.data(), n_fl, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(base + b.o_rhist, ones.data(), n_hist, cudaMemcpyHostToDevice, s));
  }
  CUDA_TRY(cudaMemcpyAsync(pending, &groups, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  dev = ResItemDev{};
  dev.inst = bi;
  dev.inst.wy = 0;
  dev.jobs = (const BatchJob *)(base + b.o_jobs);
  dev.tiles = (const TileDesc *)(base + b.o_tiles);
  dev.counters = (int32_t *)(base + b.o_cnt);
  dev.rinst = groups > 0 ? (RefineInst *)(base + b.o_rinst) : nullptr;
  dev.pending = pending;
  dev.m = it.m;
  dev.nchains = b.nchains;
  dev.ngroups = groups;
  dev.nt = p.nt;
  return TSQR_OK;
}

// ------------------------------------------------------------ reusable batch plans
// A batch planned once and replayed as a CUDA graph: the tables are uploaded at creation,
// and one run is the captured sequence of batch_enqueue plus the status and history
// copies into pinned host buffers owned by the plan.
struct tsqr_batch_plan {
  BatchBuild b;
  void *dmem = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int32_t *hstatus = nullptr;
  double *hhist = nullptr;
  cudaStream_t last = nullptr;
  bool ran = false;
};

static void plan_release(tsqr_batch_plan *P) {
  if (!P) return;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  if (P->dmem) cudaFree(P->dmem);
  if (P->hstatus) cudaFreeHost(P->hstatus);
  if (P->hhist) cudaFreeHost(P->hhist);
  delete P;
}

static tsqr_status plan_capture(tsqr_batch_plan *P, cudaStream_t cs) {
  const BatchBuild &b = P->b;
  char *base = (char *)P->dmem;
  CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  tsqr_status st = batch_enqueue(b, base, cs, false);
  if (st == TSQR_OK) {
    cudaError_t e = cudaMemcpyAsync(P->hstatus, base + b.o_st, sizeof(int32_t) * b.count, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess && !b.rinst.empty())
      e = cudaMemcpyAsync(P->hhist, base + b.o_rhist, sizeof(double) * b.max_steps * b.rinst.size(),
                          cudaMemcpyDeviceToHost, cs);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(cs, &g);  // always leave capture mode
  if (st != TSQR_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (ee != cudaSuccess) return fail(TSQR_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ee));
  P->graph = g;
  CUDA_TRY(cudaGraphInstantiate(&P->exec, g, 0));
  return TSQR_OK;
}

tsqr_status tsqr::check_batch_item(const tsqr_batch_item &it, int32_t q) {
  tsqr_status st = check_factor_args(it.A, it.m, it.n, it.lda, it.n, 2);
  if (st != TSQR_OK) return fail(st, "item %d: %s", q, g_last_error.c_str());
  if (it.prec != TSQR_FP64 && it.prec != TSQR_MIXED && it.prec != TSQR_AUTO)
    return fail(TSQR_ERR_ARG, "item %d: unknown prec", q);
  if (it.k < 0 || it.k > 64) return fail(TSQR_ERR_ARG, "item %d: k=%d outside [0, 64]", q, it.k);
  if (it.prec == TSQR_FP64 && it.n + it.k > 144)
    return fail(TSQR_ERR_ARG, "item %d: FP64 item with n + k = %d > 144", q, it.n + it.k);
  if (it.k > 0 && (!it.B || it.ldb < it.m || (it.X && it.ldx < it.n))) return fail(TSQR_ERR_ARG, "item %d: bad B/X", q);
  if (it.k > 0 && it.prec != TSQR_FP64 && !it.X) return fail(TSQR_ERR_ARG, "item %d: X is required", q);
  if (it.R && it.ldr < it.n) return fail(TSQR_ERR_ARG, "item %d: ldr < n", q);
  return TSQR_OK;
}

// FP64 or mixed for a TSQR_AUTO item by the time per row of A the cost model predicts:
// FP64 factors [A | B] (2 (n + k)^2 flops); mixed factors A in FP32 (2 n^2 flops) and
// then refines (4 n k FP64 flops per step). R-only items keep FP64 accuracy; items too
// wide to fuse B take the mixed path.
int32_t tsqr::resolve_batch_prec(const tsqr_batch_item &it) {
  if (it.prec != TSQR_AUTO) return it.prec;
  if (it.k == 0) return TSQR_FP64;
  if (it.n + it.k > 144) return TSQR_MIXED;
  const double n = it.n, k = it.k;
  const double f64 = n >= 32 ? kFp64Factor : kFp64FactorNarrow;
  const double f32 = std::min(kFp32FactorMax, kFp32FactorPerCol * n);
  const double fp64 = 2.0 * (n + k) * (n + k) / f64;
  const double fr = n >= 32 ? kRefineTflops : kRefineTflopsNarrow;
  const double mixed = 2.0 * n * n / f32 + kRefineStepsEst * 4.0 * n * k / fr;
  return mixed < fp64 ? TSQR_MIXED : TSQR_FP64;
}

size_t tsqr::batch_item_bytes(const tsqr_batch_item &it) {
  const bool mixed = resolve_batch_prec(it) == TSQR_MIXED;
  const size_t m = (size_t)it.m, n = (size_t)it.n, k = (size_t)it.k;
  if (mixed)  // FP32 chains, FP64 tree blocks, refinement partials
    return 4 * m * n + 8 * (m / 64 + 1) * n + 8 * (m / kRefineRows + 1) * n * k + n * n * 64 + 65536;
  return 8 * m * n + 8 * m * k + n * n * 64 + 65536;
}

const char *tsqr::last_error_text() { return g_last_error.c_str(); }

// Device memory a new batch can take now: what the driver reports free plus what the
// library's stream-ordered pool holds reserved but unused (it keeps freed blocks cached).
bool tsqr::debug_take_allocation_failure() {
  for (int32_t f = g_fail_allocs.load(); f > 0; f = g_fail_allocs.load())
    if (g_fail_allocs.compare_exchange_weak(f, f - 1)) return true;
  return false;
}

size_t tsqr::live_free_bytes() {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0;
  int dev = 0;
  cudaMemPool_t pool;
  if (cudaGetDevice(&dev) == cudaSuccess && lib_pool(dev, &pool) == cudaSuccess) {
    uint64_t reserved = 0, used = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
      free_b += (size_t)(reserved - used);
  }
  return free_b;
}

tsqr_status tsqr::set_last_error(tsqr_status s, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  g_last_error.vset(fmt, ap);
  va_end(ap);
  return s;
}

void tsqr::clear_last_error() { g_last_error.clear(); }

extern "C" {

static tsqr_status probe_peak(void *stream, double *tflops, double *sm_mhz, bool dmma);

tsqr_status tsqr_probe_fp64_peak(void *stream, double *tflops, double *sm_mhz) {
  return probe_peak(stream, tflops, sm_mhz, false);
}

tsqr_status tsqr_probe_dmma_peak(void *stream, double *tflops, double *sm_mhz) {
  return probe_peak(stream, tflops, sm_mhz, true);
}

static tsqr_status probe_peak(void *stream, double *tflops, double *sm_mhz, bool dmma) {
  if (!tflops) return fail(TSQR_ERR_ARG, "null output");
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  const DeviceInfo di = device_info(dev);
  if (di.sms == 0) return fail(TSQR_ERR_CUDA, "cannot query device %d", dev);
  cudaStream_t s = (cudaStream_t)stream;
  const int ctas = 4;
  double *out = nullptr;
  CUDA_TRY(pool_alloc((void **)&out, sizeof(double) * (size_t)di.sms * ctas * 256 + 64, s));
  unsigned long long *clk = (unsigned long long *)(out + (size_t)di.sms * ctas * 256);
  unsigned long long hclk[2] = {0, 0};
  double mhz = 0.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best = 0.0;
  // short launches (about 17 ms at 1.2 TFLOP/s): the burst rate, at the clock a kernel
  // timed on its own runs at; seconds of pure DFMA load would lower the clock under the
  // power cap
  const int iters = 1 << 13;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
    e = cudaEventRecord(e0, s);
    const double fl = dmma ? launch_dmma_probe(out, clk, di.sms, ctas, iters / 4, s)
                           : launch_dfma_probe(out, clk, di.sms, ctas, iters, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaMemcpy(hclk, clk, sizeof(hclk), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && rep > 0 && ms > 0.f) {
      const double tf = fl / (ms * 1e-3) / 1e12;
      if (tf > best) {
        best = tf;
        mhz = hclk[1] ? 1e3 * (double)hclk[0] / (double)hclk[1] : 0.0;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  if (e != cudaSuccess) return fail(TSQR_ERR_CUDA, "probe: %s", cudaGetErrorString(e));
  *tflops = best;
  if (sm_mhz) *sm_mhz = mhz;
  return TSQR_OK;
}

const char *tsqr_strerror(tsqr_status s) {
  switch (s) {
    case TSQR_OK: return "success";
    case TSQR_ERR_ARG: return "invalid argument";
    case TSQR_ERR_OOM: return "out of device memory";
    case TSQR_ERR_CUDA: return "CUDA error";
    case TSQR_ERR_SINGULAR: return "R is singular";
    case TSQR_ERR_TIMEOUT: return "device wait timed out";
    case TSQR_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *tsqr_last_error(void) { return g_last_error.c_str(); }

int32_t tsqr_set_mixed_wy_min_n(int32_t min_n) { return g_wy_min_n.exchange(min_n < 0 ? 0 : min_n); }

int32_t tsqr_set_apply_tile_pairs(int32_t on) { return g_tile_pairs.exchange(on ? 1 : 0); }

tsqr_status tsqr_debug_fail_allocations(int32_t count) {
  if (count < 0) return fail(TSQR_ERR_ARG, "count < 0");
  g_fail_allocs.store(count);
  return TSQR_OK;
}

tsqr_status tsqr_error_word(void *stream, int32_t *word) {
  g_last_error.clear();
  if (!word) return fail(TSQR_ERR_ARG, "word is NULL");
  int32_t *d = nullptr;
  CUDA_TRY(device_error_word(&d));
  cudaStream_t s = (cudaStream_t)stream;
  int32_t h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(int32_t), s));
  CUDA_TRY(cudaStreamSynchronize(s));
  *word = h;
  if (h & kErrTimeout) return fail(TSQR_ERR_TIMEOUT, "a bounded device wait gave up (error word 0x%x)", h);
  return TSQR_OK;
}

}  // extern "C"

// The factorization's launches on s; with QB, also Q^T QB on a helper stream of the
// device: launch q of the apply waits (event) for launch q of the factorization, so the
// apply's chain launch runs while the factorization's latency-bound tree levels leave SMs
// idle. s waits for the helper stream before the sign fix of QB.
static tsqr_status factor_common(const double *A, int64_t m, int32_t n, int64_t lda, int32_t leaf_h, int32_t arity,
                                 int32_t prec, int32_t flags, cudaStream_t s, tsqr_factors **F, double *R,
                                 int64_t ldr, double *QB, int64_t ldqb, int32_t kqb) {
  tsqr_status st = check_factor_args(A, m, n, lda, leaf_h, arity);
  if (st != TSQR_OK) return st;
  if (!F) return fail(TSQR_ERR_ARG, "F is NULL");
  if (R && ldr < n) return fail(TSQR_ERR_ARG, "ldr=%lld < n=%d", (long long)ldr, n);
  if (flags & ~(TSQR_INPLACE | TSQR_TWO_LEVEL | TSQR_CLUSTER)) return fail(TSQR_ERR_ARG, "unknown flags 0x%x", flags);
  if (prec == TSQR_MIXED) return fail(TSQR_ERR_UNSUPPORTED, "tsqr_factor: TSQR_MIXED is served by tsqr_lstsq");
  if (prec != TSQR_FP64) return fail(TSQR_ERR_ARG, "unknown prec %d", prec);
  *F = nullptr;
  tsqr_factors *f = new (std::nothrow) tsqr_factors();
  if (!f) return fail(TSQR_ERR_OOM, "host allocation failed");
  f->stream = s;
  cudaGetDevice(&f->device);
  st = get_plan(m, n, n, leaf_h, arity, flags, f->dp);
  if (st == TSQR_OK) st = factors_alloc(f, s);
  if (st == TSQR_OK) {
    if (flags & TSQR_INPLACE) {
      f->V = const_cast<double *>(A);
      f->ldv = lda;
    } else {
      cudaError_t e = pool_alloc((void **)&f->V, sizeof(double) * (size_t)m * n, s);
      if (e != cudaSuccess) st = fail(TSQR_ERR_OOM, "V allocation failed: %s", cudaGetErrorString(e));
      f->owns_V = true;
      f->ldv = m;
    }
  }
  if (st == TSQR_OK && !QB) st = run_factor(f, A, lda, nullptr, 0, s);
  if (st == TSQR_OK && QB) {
    cudaStream_t hs = helper_stream(f->device);
    if (!hs) st = fail(TSQR_ERR_CUDA, "no helper stream");
    const Plan &pl = f->plan();
    const int nl = pl.factor_launches();
    std::vector<cudaEvent_t> ev(nl + 1, nullptr);
    cudaError_t e = cudaSuccess;
    for (int q = 0; q <= nl && e == cudaSuccess && st == TSQR_OK; ++q)
      e = cudaEventCreateWithFlags(&ev[q], cudaEventDisableTiming);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "event creation: %s", cudaGetErrorString(e));
    // the helper stream starts after everything already enqueued on s (QB's producers)
    bool forked = false;
    if (st == TSQR_OK) {
      e = cudaEventRecord(ev[nl], s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(hs, ev[nl], 0);
      if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "helper stream fork: %s", cudaGetErrorString(e));
      forked = e == cudaSuccess;
    }
    FactorParams p{};
    p.A = A;
    p.lda = lda;
    p.V = f->V;
    p.ldv = f->ldv;
    p.jobs = f->dp->jobs;
    p.tiles = f->dp->tiles;
    p.tau = f->tau;
    p.scl = f->scl;
    p.n = pl.n;
    p.nc = pl.n;
    p.ldt = pl.tile_h;
    set_bounds(f, p);
    const int group = apply_group(kqb);
    for (int q = 0; q < nl && st == TSQR_OK; ++q) {
      e = factor_launch(f, p, q, s);
      if (e == cudaSuccess) e = cudaEventRecord(ev[q], s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(hs, ev[q], 0);
      if (e != cudaSuccess) {
        st = fail(TSQR_ERR_CUDA, "factor launch %d: %s", q, cudaGetErrorString(e));
        break;
      }
      int lo = 0, hi = 0;
      factor_launch_levels(pl, q, lo, hi);
      for (int li = lo; li <= hi && st == TSQR_OK; ++li)
        for (int c0 = 0; c0 < kqb && st == TSQR_OK; c0 += group)
          st = apply_launch(f, QB, ldqb, c0, std::min(group, kqb - c0), 1, 0, li, hs);
    }
    // joined even after a failed launch: the factor set's buffers are freed in the order
    // of s, after whatever the helper stream still reads
    if (forked) {
      e = cudaEventRecord(ev[nl], hs);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[nl], 0);
      if (e != cudaSuccess && st == TSQR_OK)
        st = fail(TSQR_ERR_CUDA, "helper stream join: %s", cudaGetErrorString(e));
    }
    for (cudaEvent_t x : ev)
      if (x) cudaEventDestroy(x);
  }
  if (st == TSQR_OK) {
    ProfScope ps(TSQR_PROF_SMALL, s);
    cudaError_t e = launch_extract_r(f->V, f->ldv, n, R, ldr, f->d, s);
    if (e == cudaSuccess && QB) e = launch_scale_rows(QB, ldqb, n, kqb, f->d, s);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "extract_r: %s", cudaGetErrorString(e));
  }
  if (st != TSQR_OK) {
    factors_release(f);
    return st;
  }
  *F = f;
  return TSQR_OK;
}

// B <- Q^T B (trans) or B <- Q B of F: the TSQR launches with the sign fix D, or, for a
// CAQR factor set, its panels in order (Q^T: panel 0 first; each panel acts on rows
// p*panel..m-1 of B).
static tsqr_status apply_impl(const tsqr_factors *F, double *B, int64_t ldb, int32_t k, int trans,
                              cudaStream_t s) {
  if (F->caqr()) {
    const int np = (int)F->panels.size();
    for (int i = 0; i < np; ++i) {
      const int p = trans ? i : np - 1 - i;
      tsqr_status st = apply_impl(F->panels[p], B + (int64_t)p * F->panel, ldb, k, trans, s);
      if (st != TSQR_OK) return st;
    }
    return TSQR_OK;
  }
  if (trans) {
    tsqr_status st = run_apply(F, B, ldb, k, 1, 0, s);
    if (st != TSQR_OK) return st;
    ProfScope ps(TSQR_PROF_SMALL, s);
    CUDA_TRY(launch_scale_rows(B, ldb, F->plan().n, k, F->d, s));
    return TSQR_OK;
  }
  {
    ProfScope ps(TSQR_PROF_SMALL, s);
    CUDA_TRY(launch_scale_rows(B, ldb, F->plan().n, k, F->d, s));
  }
  return run_apply(F, B, ldb, k, 0, 0, s);
}

// The thin Q of F. For CAQR, Q [I_n; 0] = Q_0 Q_1 ... Q_{P-1} [I_n; 0] is built from the
// last panel back: panel p forms its own thin Q in its columns (rows p*panel..m-1; later
// panels never touch these columns) and applies Q_p to the later panels' columns, whose
// rows p*panel..(p+1)*panel-1 are still zero. Rows above each panel's block are zero.
static tsqr_status form_q_impl(const tsqr_factors *F, double *Q, int64_t ldq, cudaStream_t s) {
  if (F->caqr()) {
    const int np = (int)F->panels.size();
    const int64_t b = F->panel;
    for (int p = 1; p < np; ++p) {
      const int64_t c0 = p * b;
      CUDA_TRY(cudaMemset2DAsync(Q + c0 * ldq, sizeof(double) * ldq, 0, sizeof(double) * c0,
                                 (size_t)F->panels[p]->plan().n, s));
    }
    for (int p = np - 1; p >= 0; --p) {
      const int64_t c0 = p * b;
      const int32_t bp = F->panels[p]->plan().n;
      const int32_t kt = F->ncols - (int32_t)c0 - bp;
      double *Qp = Q + c0 + c0 * ldq;
      if (kt > 0) {
        tsqr_status st = apply_impl(F->panels[p], Qp + (int64_t)bp * ldq, ldq, kt, 0, s);
        if (st != TSQR_OK) return st;
      }
      tsqr_status st = form_q_impl(F->panels[p], Qp, ldq, s);
      if (st != TSQR_OK) return st;
    }
    return TSQR_OK;
  }
  {
    ProfScope ps(TSQR_PROF_SMALL, s);
    CUDA_TRY(launch_formq_init(Q, ldq, F->plan().n, F->d, s));
  }
  return run_apply(F, Q, ldq, F->plan().n, 0, 1, s);
}

// ------------------------------------------------------------------------ CAQR
// Communication-avoiding QR of a wider matrix (paper §2.4; the switch from TSQR to CAQR
// for large n of §6 and Property 5 of §4): the columns are split into panels, each panel
// is factored by TSQR and its Q^T is applied to the trailing columns, whose top rows are
// rows of R; the next panel is the updated trailing block below them.
constexpr int32_t kCaqrMaxCols = 4096;  // the back substitution keeps a column of X in shared memory
constexpr int32_t kCaqrPanel = 64;      // default panel width: the TSQR kernels' widest efficient tile

static tsqr_status check_caqr_args(const double *A, int64_t m, int32_t n, int64_t lda, int32_t panel,
                                   int32_t leaf_h, int32_t arity) {
  if (!A) return fail(TSQR_ERR_ARG, "A is NULL");
  if (n < 1 || n > kCaqrMaxCols) return fail(TSQR_ERR_ARG, "n=%d outside [1, %d]", n, kCaqrMaxCols);
  if (m < n) return fail(TSQR_ERR_ARG, "m=%lld < n=%d", (long long)m, n);
  if (lda < m) return fail(TSQR_ERR_ARG, "lda=%lld < m=%lld", (long long)lda, (long long)m);
  if (panel < 0 || panel > 128) return fail(TSQR_ERR_ARG, "panel=%d outside [0, 128]", panel);
  const int32_t b = std::min(n, panel > 0 ? panel : kCaqrPanel);
  if (leaf_h < b) return fail(TSQR_ERR_ARG, "leaf_h=%d < panel width %d", leaf_h, b);
  if (!(arity == 0 || (arity >= 2 && arity <= 16))) return fail(TSQR_ERR_ARG, "arity=%d not in {0, 2..16}", arity);
  return TSQR_OK;
}

static tsqr_status caqr_factor(const double *A, int64_t m, int32_t n, int64_t lda, int32_t panel, int32_t leaf_h,
                               int32_t arity, int32_t flags, cudaStream_t s, tsqr_factors **F, double *R,
                               int64_t ldr) {
  tsqr_status st = check_caqr_args(A, m, n, lda, panel, leaf_h, arity);
  if (st != TSQR_OK) return st;
  if (!F) return fail(TSQR_ERR_ARG, "F is NULL");
  if (R && ldr < n) return fail(TSQR_ERR_ARG, "ldr=%lld < n=%d", (long long)ldr, n);
  if (flags & ~(TSQR_INPLACE | TSQR_TWO_LEVEL | TSQR_CLUSTER)) return fail(TSQR_ERR_ARG, "unknown flags 0x%x", flags);
  *F = nullptr;
  const int32_t b = panel > 0 ? panel : kCaqrPanel;
  tsqr_factors *f = new (std::nothrow) tsqr_factors();
  if (!f) return fail(TSQR_ERR_OOM, "host allocation failed");
  f->stream = s;
  cudaGetDevice(&f->device);
  f->panel = b;
  f->ncols = n;
  f->mrows = m;
  try {
    f->panels.reserve((size_t)((n + b - 1) / b));
  } catch (const std::bad_alloc &) {
    delete f;
    return fail(TSQR_ERR_OOM, "host allocation failed");
  }
  // the working copy holds every panel's reflectors and the trailing updates
  cudaError_t e = cudaSuccess;
  if (flags & TSQR_INPLACE) {
    f->V = const_cast<double *>(A);
    f->ldv = lda;
  } else {
    e = pool_alloc((void **)&f->V, sizeof(double) * (size_t)m * n, s);
    if (e == cudaSuccess) {
      f->owns_V = true;
      f->ldv = m;
      e = cudaMemcpy2DAsync(f->V, sizeof(double) * m, A, sizeof(double) * lda, sizeof(double) * m, n,
                            cudaMemcpyDeviceToDevice, s);
    }
  }
  if (e == cudaSuccess) e = pool_alloc((void **)&f->Rfull, sizeof(double) * (size_t)n * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->Rfull, 0, sizeof(double) * (size_t)n * n, s);
  if (e != cudaSuccess) st = fail(TSQR_ERR_OOM, "CAQR workspace: %s", cudaGetErrorString(e));
  for (int32_t c0 = 0; c0 < n && st == TSQR_OK; c0 += b) {
    const int32_t bp = std::min(b, n - c0);
    const int32_t kt = n - c0 - bp;  // trailing columns
    double *Wp = f->V + c0 + (int64_t)c0 * f->ldv;
    double *Tp = kt > 0 ? Wp + (int64_t)bp * f->ldv : nullptr;
    tsqr_factors *fp = nullptr;
    // the panel in place in the working copy; Q_p^T of the trailing columns overlaps the
    // panel's reduction tree (tsqr_factor_qt's launch pairing)
    st = factor_common(Wp, m - c0, bp, f->ldv, leaf_h, arity, TSQR_FP64, (flags & (TSQR_TWO_LEVEL | TSQR_CLUSTER)) | TSQR_INPLACE, s,
                       &fp, f->Rfull + c0 + (int64_t)c0 * n, n, Tp, f->ldv, kt);
    if (st != TSQR_OK) break;
    f->panels.push_back(fp);
    if (kt > 0) {  // rows c0..c0+bp-1 of the updated trailing columns are rows of R (diag(R) >= 0 signs)
      e = cudaMemcpy2DAsync(f->Rfull + c0 + (int64_t)(c0 + bp) * n, sizeof(double) * n, Tp,
                            sizeof(double) * f->ldv, sizeof(double) * bp, kt, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "R row copy: %s", cudaGetErrorString(e));
    }
  }
  if (st == TSQR_OK && R) {
    e = cudaMemcpy2DAsync(R, sizeof(double) * ldr, f->Rfull, sizeof(double) * n, sizeof(double) * n, n,
                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "R copy: %s", cudaGetErrorString(e));
  }
  if (st != TSQR_OK) {
    factors_release(f);
    return st;
  }
  *F = f;
  return TSQR_OK;
}

// Least squares through CAQR (n > 128): X = R^{-1} (Q^T B)[0:n], FP64 only.
static tsqr_status caqr_lstsq(const double *A, int64_t m, int32_t n, int64_t lda, const double *B, int64_t ldb,
                              int32_t k, double *X, int64_t ldx, int32_t leaf_h, int32_t arity, int32_t prec,
                              int32_t flags, cudaStream_t s, double *info) {
  tsqr_status st = check_caqr_args(A, m, n, lda, 0, leaf_h, arity);
  if (st != TSQR_OK) return st;
  if (!B || !X) return fail(TSQR_ERR_ARG, "B or X is NULL");
  if (k < 1 || k > 64) return fail(TSQR_ERR_ARG, "k=%d outside [1, 64]", k);
  if (ldb < m || ldx < n) return fail(TSQR_ERR_ARG, "bad ldb/ldx");
  if (flags & ~(TSQR_INPLACE | TSQR_TWO_LEVEL | TSQR_CLUSTER)) return fail(TSQR_ERR_ARG, "unknown flags 0x%x", flags);
  if (prec == TSQR_MIXED) return fail(TSQR_ERR_UNSUPPORTED, "TSQR_MIXED least squares takes n <= 128");
  if (prec != TSQR_FP64) return fail(TSQR_ERR_ARG, "unknown prec %d", prec);
  tsqr_factors *F = nullptr;
  st = caqr_factor(A, m, n, lda, 0, leaf_h, arity, flags & (TSQR_TWO_LEVEL | TSQR_CLUSTER), s, &F, nullptr, 0);
  if (st != TSQR_OK) return st;
  double *W = nullptr;  // Q^T B workspace (m-by-k)
  int32_t *status = nullptr;
  cudaError_t e = pool_alloc((void **)&W, sizeof(double) * (size_t)m * k, s);
  if (e == cudaSuccess) e = pool_alloc((void **)&status, sizeof(int32_t), s);
  if (e != cudaSuccess) st = fail(TSQR_ERR_OOM, "workspace allocation failed");
  if (st == TSQR_OK) {
    e = cudaMemcpy2DAsync(W, sizeof(double) * m, B, sizeof(double) * ldb, sizeof(double) * m, k,
                          cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "workspace init: %s", cudaGetErrorString(e));
  }
  if (st == TSQR_OK) st = apply_impl(F, W, m, k, 1, s);
  if (st == TSQR_OK) {
    ProfScope ps(TSQR_PROF_SMALL, s);
    e = launch_trsv(F->Rfull, n, n, W, m, k, X, ldx, nullptr, status, s);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "trsv: %s", cudaGetErrorString(e));
  }
  int32_t hstatus = 0;
  if (st == TSQR_OK) {
    e = cudaMemcpyAsync(&hstatus, status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "status readback: %s", cudaGetErrorString(e));
  }
  if (st == TSQR_OK && info) info[0] = 0.0;
  if (W) cudaFreeAsync(W, s);
  if (status) cudaFreeAsync(status, s);
  factors_release(F);
  if (st == TSQR_OK && hstatus == 4) return fail(TSQR_ERR_SINGULAR, "R has a zero diagonal entry");
  return st;
}

extern "C" {

tsqr_status tsqr_factor(const double *A, int64_t m, int32_t n, int64_t lda, int32_t leaf_h, int32_t arity,
                        int32_t prec, int32_t flags, void *stream, tsqr_factors **F, double *R, int64_t ldr) {
  g_last_error.clear();
  return factor_common(A, m, n, lda, leaf_h, arity, prec, flags, (cudaStream_t)stream, F, R, ldr, nullptr, 0, 0);
}

tsqr_status tsqr_factor_qt(const double *A, int64_t m, int32_t n, int64_t lda, double *B, int64_t ldb, int32_t k,
                           int32_t leaf_h, int32_t arity, int32_t prec, int32_t flags, void *stream,
                           tsqr_factors **F, double *R, int64_t ldr) {
  g_last_error.clear();
  if (!B || k < 1 || ldb < m) return fail(TSQR_ERR_ARG, "bad B, k=%d or ldb=%lld", k, (long long)ldb);
  if (flags & TSQR_INPLACE) return fail(TSQR_ERR_ARG, "tsqr_factor_qt: TSQR_INPLACE is not supported");
  return factor_common(A, m, n, lda, leaf_h, arity, prec, flags, (cudaStream_t)stream, F, R, ldr, B, ldb, k);
}

tsqr_status tsqr_apply_qt(const tsqr_factors *F, double *B, int64_t ldb, int32_t k, void *stream) {
  g_last_error.clear();
  if (!F || !B) return fail(TSQR_ERR_ARG, "NULL factor set or B");
  if (k < 1 || ldb < F->rows()) return fail(TSQR_ERR_ARG, "bad k=%d or ldb=%lld", k, (long long)ldb);
  return apply_impl(F, B, ldb, k, 1, (cudaStream_t)stream);
}

tsqr_status tsqr_apply_q(const tsqr_factors *F, double *B, int64_t ldb, int32_t k, void *stream) {
  g_last_error.clear();
  if (!F || !B) return fail(TSQR_ERR_ARG, "NULL factor set or B");
  if (k < 1 || ldb < F->rows()) return fail(TSQR_ERR_ARG, "bad k=%d or ldb=%lld", k, (long long)ldb);
  return apply_impl(F, B, ldb, k, 0, (cudaStream_t)stream);
}

tsqr_status tsqr_form_q(const tsqr_factors *F, double *Q, int64_t ldq, void *stream) {
  g_last_error.clear();
  if (!F || !Q) return fail(TSQR_ERR_ARG, "NULL factor set or Q");
  if (ldq < F->rows()) return fail(TSQR_ERR_ARG, "ldq=%lld < m", (long long)ldq);
  return form_q_impl(F, Q, ldq, (cudaStream_t)stream);
}

tsqr_status tsqr_caqr(const double *A, int64_t m, int32_t n, int64_t lda, int32_t panel, int32_t leaf_h,
                      int32_t arity, int32_t flags, void *stream, tsqr_factors **F, double *R, int64_t ldr) {
  g_last_error.clear();
  return caqr_factor(A, m, n, lda, panel, leaf_h, arity, flags, (cudaStream_t)stream, F, R, ldr);
}

tsqr_status tsqr_orthonormalize(const double *A, int64_t m, int32_t n, int64_t lda, double *Q, int64_t ldq,
                                double *R, int64_t ldr, int32_t leaf_h, int32_t arity, int32_t prec,
                                int32_t flags, void *stream) {
  g_last_error.clear();
  if (!Q || ldq < m) return fail(TSQR_ERR_ARG, "NULL Q or ldq=%lld < m=%lld", (long long)ldq, (long long)m);
  if (flags & TSQR_INPLACE) return fail(TSQR_ERR_ARG, "tsqr_orthonormalize: TSQR_INPLACE is not supported");
  cudaStream_t s = (cudaStream_t)stream;
  tsqr_factors *F = nullptr;
  tsqr_status st;
  if (n > 128) {  // CAQR with the default panel width
    if (prec != TSQR_FP64) return fail(prec == TSQR_MIXED ? TSQR_ERR_UNSUPPORTED : TSQR_ERR_ARG, "prec %d", prec);
    st = caqr_factor(A, m, n, lda, 0, leaf_h, arity, flags, s, &F, R, ldr);
  } else {
    st = factor_common(A, m, n, lda, leaf_h, arity, prec, flags, s, &F, R, ldr, nullptr, 0, 0);
  }
  if (st != TSQR_OK) return st;
  // the factorization has read all of A before the first write to Q (stream order), and
  // V is the factor set's own copy, so Q may alias A
  st = form_q_impl(F, Q, ldq, s);
  factors_release(F);
  return st;
}

tsqr_status tsqr_solve_r(const tsqr_factors *F, const double *C, int64_t ldc, int32_t k, double *X, int64_t ldx,
                         int32_t *status, void *stream) {
  g_last_error.clear();
  if (!F || !C || !X) return fail(TSQR_ERR_ARG, "NULL factor set, C or X");
  const int n = F->cols();
  if (k < 1 || ldc < n || ldx < n) return fail(TSQR_ERR_ARG, "bad k=%d, ldc or ldx", k);
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope ps(TSQR_PROF_SMALL, s);
  if (F->caqr())
    CUDA_TRY(launch_trsv(F->Rfull, n, n, C, ldc, k, X, ldx, nullptr, status, s));
  else
    CUDA_TRY(launch_trsv(F->V, F->ldv, n, C, ldc, k, X, ldx, F->d, status, s));
  return TSQR_OK;
}

tsqr_status tsqr_lstsq(const double *A, int64_t m, int32_t n, int64_t lda, const double *B, int64_t ldb,
                       int32_t k, double *X, int64_t ldx, int32_t leaf_h, int32_t arity, int32_t prec,
                       int32_t flags, int32_t max_refine, void *stream, double *info) {
  g_last_error.clear();
  if (n > 128)
    return caqr_lstsq(A, m, n, lda, B, ldb, k, X, ldx, leaf_h, arity, prec, flags, (cudaStream_t)stream, info);
  tsqr_status st = check_factor_args(A, m, n, lda, leaf_h, arity);
  if (st != TSQR_OK) return st;
  if (!B || !X) return fail(TSQR_ERR_ARG, "B or X is NULL");
  if (k < 1 || k > 64) return fail(TSQR_ERR_ARG, "k=%d outside [1, 64]", k);
  if (ldb < m || ldx < n) return fail(TSQR_ERR_ARG, "bad ldb/ldx");
  if (flags & ~(TSQR_INPLACE | TSQR_TWO_LEVEL | TSQR_CLUSTER)) return fail(TSQR_ERR_ARG, "unknown flags 0x%x", flags);
  if (max_refine < 0) return fail(TSQR_ERR_ARG, "max_refine < 0");
  if (prec != TSQR_FP64 && prec != TSQR_MIXED) return fail(TSQR_ERR_ARG, "unknown prec %d", prec);
  flags &= ~TSQR_INPLACE;
  if (prec == TSQR_MIXED) {
    tsqr_batch_item it{};
    it.A = A;
    it.m = m;
    it.n = n;
    it.lda = lda;
    it.B = B;
    it.ldb = ldb;
    it.k = k;
    it.X = X;
    it.ldx = ldx;
    it.prec = TSQR_MIXED;
    try {
      return lstsq_mixed_batched(it, arity == 0 ? 2 : arity, max_refine + 1, (cudaStream_t)stream, info);
    } catch (const std::bad_alloc &) {
      return fail(TSQR_ERR_OOM, "host allocation failed");
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  tsqr_factors *f = new (std::nothrow) tsqr_factors();
  if (!f) return fail(TSQR_ERR_OOM, "host allocation failed");
  f->stream = s;
  double *W = nullptr;  // Q^T B workspace (m-by-k)
  int32_t *status = nullptr;
  const bool fused = (n + k) <= 128;
  st = get_plan(m, n, fused ? n + k : n, leaf_h, arity, flags, f->dp);
  if (st == TSQR_OK) st = factors_alloc(f, s);
  if (st == TSQR_OK) {
    cudaError_t e = pool_alloc((void **)&f->V, sizeof(double) * (size_t)m * n, s);
    if (e == cudaSuccess) e = pool_alloc((void **)&W, sizeof(double) * (size_t)m * k, s);
    if (e == cudaSuccess) e = pool_alloc((void **)&status, sizeof(int32_t), s);
    if (e != cudaSuccess) st = fail(TSQR_ERR_OOM, "workspace allocation failed");
    f->owns_V = true;
    f->ldv = m;
  }
  if (st == TSQR_OK) {
    cudaError_t e = cudaMemcpy2DAsync(W, sizeof(double) * m, B, sizeof(double) * ldb, sizeof(double) * m, k,
                                      cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "workspace init: %s", cudaGetErrorString(e));
  }
  if (st == TSQR_OK) {
    if (fused) {
      st = run_factor(f, A, lda, W, m, s);  // Q^T B computed with the factorization
    } else {
      st = run_factor(f, A, lda, nullptr, 0, s);
      if (st == TSQR_OK) st = run_apply(f, W, m, k, 1, 0, s);
    }
  }
  if (st == TSQR_OK) {
    ProfScope ps(TSQR_PROF_SMALL, s);
    cudaError_t e = launch_trsv(f->V, f->ldv, n, W, m, k, X, ldx, nullptr, status, s);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "trsv: %s", cudaGetErrorString(e));
  }
  int32_t hstatus = 0;
  if (st == TSQR_OK) {
    cudaError_t e = cudaMemcpyAsync(&hstatus, status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "status readback: %s", cudaGetErrorString(e));
  }
  if (st == TSQR_OK && info) info[0] = 0.0;
  if (W) cudaFreeAsync(W, s);
  if (status) cudaFreeAsync(status, s);
  factors_release(f);
  if (st == TSQR_OK && hstatus == 4) return fail(TSQR_ERR_SINGULAR, "R has a zero diagonal entry");
  return st;
}


// A column-major block copy: one linear copy when both leading dimensions equal the rows.
static cudaError_t copy_block(double *dst, int64_t ldd, const double *src, int64_t lds, int64_t rows, int64_t cols,
                              cudaMemcpyKind kind, cudaStream_t s) {
  if (ldd == rows && lds == rows) return cudaMemcpyAsync(dst, src, sizeof(double) * rows * cols, kind, s);
  return cudaMemcpy2DAsync(dst, sizeof(double) * ldd, src, sizeof(double) * lds, sizeof(double) * rows, cols, kind, s);
}

tsqr_status tsqr_qr_solve_host(const double *A, int64_t m, int32_t n, int64_t lda, const double *B, int64_t ldb,
                               int32_t k, double *Q, int64_t ldq, double *R, int64_t ldr, double *X, int64_t ldx,
                               int32_t *status, int32_t leaf_h, int32_t arity, int32_t flags, void *stream,
                               void *after, void *done) {
  g_last_error.clear();
  tsqr_status st = check_factor_args(A, m, n, lda, leaf_h, arity);
  if (st != TSQR_OK) return st;
  if ((B == nullptr) != (X == nullptr)) return fail(TSQR_ERR_ARG, "B and X go together");
  if (B && (k < 1 || ldb < m || ldx < n)) return fail(TSQR_ERR_ARG, "bad k=%d, ldb or ldx", k);
  if (Q && ldq < m) return fail(TSQR_ERR_ARG, "ldq=%lld < m", (long long)ldq);
  if (R && ldr < n) return fail(TSQR_ERR_ARG, "ldr=%lld < n", (long long)ldr);
  if (flags & ~(TSQR_TWO_LEVEL | TSQR_CLUSTER)) return fail(TSQR_ERR_ARG, "unknown flags 0x%x", flags);
  if (!B) k = 0;
  cudaStream_t s = (cudaStream_t)stream;
  // device copies of the inputs and outputs, from the stream-ordered pool
  double *Ad = nullptr, *Bd = nullptr, *Qd = nullptr, *Rd = nullptr, *Xd = nullptr;
  int32_t *sd = nullptr;
  cudaError_t e = pool_alloc((void **)&Ad, sizeof(double) * (size_t)m * n, s);
  if (e == cudaSuccess && B) e = pool_alloc((void **)&Bd, sizeof(double) * (size_t)m * k, s);
  if (e == cudaSuccess && B) e = pool_alloc((void **)&Xd, sizeof(double) * (size_t)n * k, s);
  if (e == cudaSuccess && Q) e = pool_alloc((void **)&Qd, sizeof(double) * (size_t)m * n, s);
  if (e == cudaSuccess) e = pool_alloc((void **)&Rd, sizeof(double) * (size_t)n * n, s);
  if (e == cudaSuccess) e = pool_alloc((void **)&sd, sizeof(int32_t), s);
  if (e != cudaSuccess) st = fail(TSQR_ERR_OOM, "device buffers: %s", cudaGetErrorString(e));
  if (st == TSQR_OK) {
    e = copy_block(Ad, m, A, lda, m, n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && B) e = copy_block(Bd, m, B, ldb, m, k, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sd, 0, sizeof(int32_t), s);
    if (e == cudaSuccess && after) e = cudaStreamWaitEvent(s, (cudaEvent_t)after, 0);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "input copies: %s", cudaGetErrorString(e));
  }
  tsqr_factors *F = nullptr;
  if (st == TSQR_OK) st = factor_common(Ad, m, n, m, leaf_h, arity, TSQR_FP64, flags, s, &F, Rd, n, nullptr, 0, 0);
  // Q^T B and the back substitution on the library's helper stream, beside the thin Q
  cudaStream_t hs = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  bool forked = false;
  if (st == TSQR_OK && B) {
    hs = helper_stream(F->device);
    e = hs ? cudaSuccess : cudaErrorNotReady;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hs, ev[0], 0);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "helper stream fork: %s", cudaGetErrorString(e));
    forked = st == TSQR_OK;
    if (st == TSQR_OK) st = apply_impl(F, Bd, m, k, 1, hs);
    if (st == TSQR_OK) {
      ProfScope ps(TSQR_PROF_SMALL, hs);
      e = launch_trsv(F->V, F->ldv, n, Bd, m, k, Xd, n, F->d, sd, hs);
      if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "trsv: %s", cudaGetErrorString(e));
    }
  }
  if (st == TSQR_OK && Q) st = form_q_impl(F, Qd, m, s);
  if (forked) {  // joined even after a failure: the buffers are freed in the order of s
    e = cudaEventRecord(ev[1], hs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[1], 0);
    if (e != cudaSuccess && st == TSQR_OK) st = fail(TSQR_ERR_CUDA, "helper stream join: %s", cudaGetErrorString(e));
  }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  if (st == TSQR_OK && done) {
    e = cudaEventRecord((cudaEvent_t)done, s);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "done event: %s", cudaGetErrorString(e));
  }
  if (st == TSQR_OK) {
    e = cudaSuccess;
    if (Q) e = copy_block(Q, ldq, Qd, m, m, n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && R) e = copy_block(R, ldr, Rd, n, n, n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && X) e = copy_block(X, ldx, Xd, n, n, k, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && status) e = cudaMemcpyAsync(status, sd, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "output copies: %s", cudaGetErrorString(e));
  }
  if (F) factors_release(F);
  for (void *b : {(void *)Ad, (void *)Bd, (void *)Qd, (void *)Rd, (void *)Xd, (void *)sd})
    if (b) cudaFreeAsync(b, s);
  return st;
}

tsqr_status tsqr_batch_plan_create(const tsqr_batch_item *items, int32_t count, int32_t chain_tiles, int32_t arity,
                                   tsqr_batch_plan **out) {
  g_last_error.clear();
  if (!out) return fail(TSQR_ERR_ARG, "null plan pointer");
  *out = nullptr;
  if (count < 1 || !items) return fail(TSQR_ERR_ARG, "bad items/count");
  if (chain_tiles < 0 || !(arity == 0 || (arity >= 2 && arity <= 16))) return fail(TSQR_ERR_ARG, "bad chain_tiles/arity");
  for (int32_t q = 0; q < count; ++q) {
    tsqr_status st = check_batch_item(items[q], q);
    if (st != TSQR_OK) return st;
  }
  tsqr_batch_plan *P = nullptr;
  try {
    P = new tsqr_batch_plan();
    tsqr_status st = batch_build(items, count, chain_tiles, arity, P->b);
    if (st != TSQR_OK) {
      plan_release(P);
      return st;
    }
  } catch (const std::bad_alloc &) {
    plan_release(P);
    return fail(TSQR_ERR_OOM, "host allocation failed");
  }
  cudaStream_t cs = nullptr;
  auto bail = [&](tsqr_status st) {
    if (cs) cudaStreamDestroy(cs);
    plan_release(P);
    return st;
  };
  cudaError_t e = cudaMalloc(&P->dmem, P->b.bytes);
  if (e != cudaSuccess) return bail(fail(TSQR_ERR_OOM, "plan workspace of %zu bytes: %s", P->b.bytes, cudaGetErrorString(e)));
  e = cudaMallocHost(&P->hstatus, sizeof(int32_t) * count);
  if (e == cudaSuccess && !P->b.rinst.empty())
    e = cudaMallocHost(&P->hhist, sizeof(double) * P->b.max_steps * P->b.rinst.size());
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(fail(TSQR_ERR_CUDA, "plan setup: %s", cudaGetErrorString(e)));
  batch_bind(P->b, (char *)P->dmem);
  tsqr_status st = batch_upload(P->b, (char *)P->dmem, cs);
  if (st == TSQR_OK) {
    e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "plan upload: %s", cudaGetErrorString(e));
  }
  if (st == TSQR_OK) st = plan_capture(P, cs);
  if (st != TSQR_OK) return bail(st);
  cudaStreamDestroy(cs);
  *out = P;
  return TSQR_OK;
}

tsqr_status tsqr_batch_plan_run(tsqr_batch_plan *P, void *stream) {
  if (!P) return fail(TSQR_ERR_ARG, "null plan");
  CUDA_TRY(cudaGraphLaunch(P->exec, (cudaStream_t)stream));
  P->last = (cudaStream_t)stream;
  P->ran = true;
  return TSQR_OK;
}

tsqr_status tsqr_batch_plan_results(tsqr_batch_plan *P, int32_t *status, double *info) {
  if (!P) return fail(TSQR_ERR_ARG, "null plan");
  if (!P->ran) return fail(TSQR_ERR_ARG, "the plan has not run");
  CUDA_TRY(cudaStreamSynchronize(P->last));
  if (status) std::copy(P->hstatus, P->hstatus + P->b.count, status);
  if (info) {
    if (P->b.rinst.empty())
      std::fill(info, info + 2 * P->b.count, 0.0);
    else
      batch_info(P->b, P->hhist, info);
  }
  return TSQR_OK;
}

tsqr_status tsqr_batch_plan_destroy(tsqr_batch_plan *P) {
  if (!P) return TSQR_OK;
  if (P->ran) cudaStreamSynchronize(P->last);
  plan_release(P);
  return TSQR_OK;
}

// ------------------------------------------------------------------- autotuners
// Both time their candidates with CUDA events on the caller's stream, on the caller's
// own data, and return the fastest; each candidate runs once untimed first (planning,
// pool growth) and then twice timed, keeping the faster run.
namespace {
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};
}  // namespace

tsqr_status tsqr_batch_autotune(const tsqr_batch_item *items, int32_t count, int32_t sample, void *stream,
                                int32_t *chain_tiles, int32_t *arity, float *ms_table) {
  g_last_error.clear();
  if (count < 1 || !items || !chain_tiles || !arity) return fail(TSQR_ERR_ARG, "bad items/count/outputs");
  for (int32_t q = 0; q < count; ++q) {
    tsqr_status st = check_batch_item(items[q], q);
    if (st != TSQR_OK) return st;
  }
  const int32_t S = sample > 0 ? std::min(sample, count) : std::min<int32_t>(count, 1000);
  cudaStream_t s = (cudaStream_t)stream;
  EventPair ev;
  CUDA_TRY(cudaEventCreate(&ev.a));
  CUDA_TRY(cudaEventCreate(&ev.b));
  float best = 0.f;
  int32_t q = 0;
  try {
    for (int32_t L : kBatchTuneChainTiles) {
      for (int32_t ar : kBatchTuneArity) {
        float t = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
          if (rep > 0) CUDA_TRY(cudaEventRecord(ev.a, s));
          tsqr_status st = batch_solve_internal(items, S, L, ar, s, nullptr, nullptr, nullptr);
          if (st != TSQR_OK) return st;
          if (rep > 0) {
            CUDA_TRY(cudaEventRecord(ev.b, s));
            CUDA_TRY(cudaEventSynchronize(ev.b));
            float ms = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&ms, ev.a, ev.b));
            t = (rep == 1) ? ms : std::min(t, ms);
          }
        }
        if (ms_table) ms_table[q] = t;
        if (q == 0 || t < best) {
          best = t;
          *chain_tiles = L;
          *arity = ar;
        }
        ++q;
      }
    }
  } catch (const std::bad_alloc &) {
    return fail(TSQR_ERR_OOM, "host allocation failed");
  }
  return TSQR_OK;
}

tsqr_status tsqr_factor_autotune(const double *A, int64_t m, int32_t n, int64_t lda, void *stream, int32_t *leaf_h,
                                 int32_t *arity, int32_t *flags, float *best_ms) {
  g_last_error.clear();
  tsqr_status st = check_factor_args(A, m, n, lda, n, 2);
  if (st != TSQR_OK) return st;
  if (!leaf_h || !arity || !flags) return fail(TSQR_ERR_ARG, "NULL output");
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  const DeviceInfo di = device_info(dev);
  if (di.sms == 0) return fail(TSQR_ERR_CUDA, "cannot query device %d", dev);
  int th = 0, cps = 0;
  if (!factor_tile_choice(n, n, 1 << 20, (size_t)di.smem_sm, (size_t)di.reserved, (size_t)di.optin, 3, th, cps))
    return fail(TSQR_ERR_UNSUPPORTED, "no tile height fits shared memory for n=%d", n);
  // candidates: the two-level tree and the pure k-ary tree over leaves of 1, 4 and 16
  // tiles; the flat tree (one chain, one CTA) only while it has at most one tile per SM
  struct Cand {
    int32_t h, ar, fl;
  };
  std::vector<Cand> cands;
  for (int32_t mult : {1, 4, 16})
    for (int32_t ar : {2, 4}) {
      cands.push_back({th * mult, ar, TSQR_TWO_LEVEL});
      cands.push_back({th * mult, ar, 0});
    }
  if ((m + th - 1) / th <= di.sms) cands.push_back({th, 0, 0});
  cudaStream_t s = (cudaStream_t)stream;
  EventPair ev;
  CUDA_TRY(cudaEventCreate(&ev.a));
  CUDA_TRY(cudaEventCreate(&ev.b));
  float best = 0.f;
  bool have = false;
  for (const Cand &c : cands) {
    if ((int64_t)c.h > m) continue;
    float t = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
      if (rep > 0) CUDA_TRY(cudaEventRecord(ev.a, s));
      tsqr_factors *F = nullptr;
      st = tsqr_factor(A, m, n, lda, c.h, c.ar, TSQR_FP64, c.fl, stream, &F, nullptr, 0);
      if (st != TSQR_OK) return st;
      tsqr_free(F);
      if (rep > 0) {
        CUDA_TRY(cudaEventRecord(ev.b, s));
        CUDA_TRY(cudaEventSynchronize(ev.b));
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, ev.a, ev.b));
        t = (rep == 1) ? ms : std::min(t, ms);
      }
    }
    if (!have || t < best) {
      have = true;
      best = t;
      *leaf_h = c.h;
      *arity = c.ar;
      *flags = c.fl;
    }
  }
  if (!have) return fail(TSQR_ERR_UNSUPPORTED, "no candidate fits m=%lld", (long long)m);
  if (best_ms) *best_ms = best;
  return TSQR_OK;
}

tsqr_status tsqr_batch_solve(const tsqr_batch_item *items, int32_t count, int32_t chain_tiles, int32_t arity,
                             void *stream, int32_t *status, double *info) {
  g_last_error.clear();
  if (count < 0 || (count > 0 && !items)) return fail(TSQR_ERR_ARG, "bad items/count");
  if (chain_tiles < 0 || !(arity == 0 || (arity >= 2 && arity <= 16))) return fail(TSQR_ERR_ARG, "bad chain_tiles/arity");
  for (int32_t q = 0; q < count; ++q) {
    tsqr_status st = check_batch_item(items[q], q);
    if (st != TSQR_OK) return st;
  }
  if (count == 0) return TSQR_OK;
  try {
    return batch_solve_internal(items, count, chain_tiles, arity, (cudaStream_t)stream, status, nullptr, info);
  } catch (const std::bad_alloc &) {
    return fail(TSQR_ERR_OOM, "host allocation failed");
  }
}

tsqr_status tsqr_free(tsqr_factors *F) {
  factors_release(F);
  return TSQR_OK;
}

tsqr_status tsqr_plan_describe(int64_t m, int32_t n, int32_t nc, int32_t leaf_h, int32_t arity, int32_t flags,
                               int32_t sms, int64_t smem_per_sm, int64_t smem_reserved, int64_t smem_optin,
                               int64_t *out, int64_t *tiles, int64_t max_tiles, int64_t *jobs,
                               int64_t max_jobs) {
  g_last_error.clear();
  int dummy = 0;
  tsqr_status st = check_factor_args(&dummy, m, n, m, leaf_h, arity);
  if (st != TSQR_OK) return st;
  if (!out) return fail(TSQR_ERR_ARG, "out is NULL");
  if (nc < n || nc > 256) return fail(TSQR_ERR_ARG, "nc=%d outside [n, 256]", nc);
  if (flags & ~(TSQR_INPLACE | TSQR_TWO_LEVEL | TSQR_CLUSTER)) return fail(TSQR_ERR_ARG, "unknown flags 0x%x", flags);
  if (sms < 1 || smem_per_sm < 1 || smem_reserved < 0 || smem_optin < 1)
    return fail(TSQR_ERR_ARG, "bad device description");
  DeviceInfo di;
  di.sms = sms;
  di.smem_sm = (size_t)smem_per_sm;
  di.reserved = (size_t)smem_reserved;
  di.optin = (size_t)smem_optin;
  Plan pl;
  st = make_plan_on(di, pl, m, n, nc, leaf_h, arity, flags);
  if (st != TSQR_OK) return st;
  plan_info(pl, out);
  if (tiles && (int64_t)pl.tiles.size() > max_tiles) return fail(TSQR_ERR_ARG, "max_tiles too small");
  if (jobs && (int64_t)pl.jobs.size() > max_jobs) return fail(TSQR_ERR_ARG, "max_jobs too small");
  for (size_t l = 0; l < pl.launches.size(); ++l) {
    const LaunchDesc &ld = pl.launches[l];
    for (int32_t jb = ld.job_begin; jb < ld.job_begin + ld.job_count; ++jb) {
      const JobDesc &jd = pl.jobs[jb];
      if (jobs) {
        jobs[4 * jb + 0] = jd.piv_row;
        jobs[4 * jb + 1] = jd.tile_begin;
        jobs[4 * jb + 2] = jd.tile_count;
        jobs[4 * jb + 3] = (int64_t)l;
      }
      if (tiles) {
        for (int32_t t = jd.tile_begin; t < jd.tile_begin + jd.tile_count; ++t) {
          tiles[5 * t + 0] = pl.tiles[t].row0;
          tiles[5 * t + 1] = pl.tiles[t].nrows;
          tiles[5 * t + 2] = pl.tiles[t].kind;
          tiles[5 * t + 3] = jb;
          tiles[5 * t + 4] = (int64_t)l;
        }
      }
    }
  }
  return TSQR_OK;
}

tsqr_status tsqr_plan_clusters(int64_t m, int32_t n, int32_t nc, int32_t leaf_h, int32_t flags, int32_t sms,
                               int64_t smem_per_sm, int64_t smem_reserved, int64_t smem_optin, int64_t *out,
                               int32_t *launches, int64_t max_launches, int32_t *slots, int64_t max_slots) {
  g_last_error.clear();
  int dummy = 0;
  tsqr_status st = check_factor_args(&dummy, m, n, m, leaf_h, 2);
  if (st != TSQR_OK) return st;
  if (!out) return fail(TSQR_ERR_ARG, "out is NULL");
  if (nc < n || nc > 256) return fail(TSQR_ERR_ARG, "nc=%d outside [n, 256]", nc);
  if (sms < 1 || smem_per_sm < 1 || smem_reserved < 0 || smem_optin < 1)
    return fail(TSQR_ERR_ARG, "bad device description");
  DeviceInfo di;
  di.sms = sms;
  di.smem_sm = (size_t)smem_per_sm;
  di.reserved = (size_t)smem_reserved;
  di.optin = (size_t)smem_optin;
  Plan pl;
  st = make_plan_on(di, pl, m, n, nc, leaf_h, 2, (flags & TSQR_TWO_LEVEL) | TSQR_CLUSTER);
  if (st != TSQR_OK) return st;
  out[0] = (int64_t)pl.cl_launches.size();
  out[1] = (int64_t)pl.cl_slots.size();
  if (launches && (int64_t)pl.cl_launches.size() > max_launches) return fail(TSQR_ERR_ARG, "max_launches too small");
  if (slots && (int64_t)pl.cl_slots.size() > max_slots) return fail(TSQR_ERR_ARG, "max_slots too small");
  for (size_t q = 0; launches && q < pl.cl_launches.size(); ++q) {
    const Plan::ClusterLaunch &cl = pl.cl_launches[q];
    launches[4 * q + 0] = cl.slot_begin;
    launches[4 * q + 1] = cl.nclusters;
    launches[4 * q + 2] = cl.level_lo;
    launches[4 * q + 3] = cl.level_hi;
  }
  for (size_t q = 0; slots && q < pl.cl_slots.size(); ++q) {
    slots[3 * q + 0] = pl.cl_slots[q].job;
    slots[3 * q + 1] = pl.cl_slots[q].child[0];
    slots[3 * q + 2] = pl.cl_slots[q].child[1];
  }
  return TSQR_OK;
}

tsqr_status tsqr_batch_describe(const tsqr_batch_item *items, int32_t count, int32_t chain_tiles, int32_t arity,
                                int32_t sms, int64_t smem_per_sm, int64_t smem_reserved, int64_t smem_optin,
                                int64_t *out, int64_t *jobs, int64_t max_jobs) {
  g_last_error.clear();
  if (!out || count < 1 || !items) return fail(TSQR_ERR_ARG, "bad items/count/out");
  if (chain_tiles < 0 || !(arity == 0 || (arity >= 2 && arity <= 16))) return fail(TSQR_ERR_ARG, "bad chain_tiles/arity");
  if (sms < 1 || smem_per_sm < 1 || smem_reserved < 0 || smem_optin < 1)
    return fail(TSQR_ERR_ARG, "bad device description");
  for (int32_t q = 0; q < count; ++q) {
    tsqr_status st = check_batch_item(items[q], q);
    if (st != TSQR_OK) return st;
  }
  DeviceInfo di;
  di.sms = sms;
  di.smem_sm = (size_t)smem_per_sm;
  di.reserved = (size_t)smem_reserved;
  di.optin = (size_t)smem_optin;
  try {
    BatchBuild b;
    tsqr_status st = batch_build_on(di, items, count, chain_tiles, arity, b, kRefineSteps, 0);
    if (st != TSQR_OK) return st;
    out[0] = b.nchains;
    out[1] = b.njobs;
    out[2] = b.ntiles;
    out[3] = b.grid;
    if (jobs && b.njobs > max_jobs) return fail(TSQR_ERR_ARG, "max_jobs too small");
    for (int32_t j = 0; jobs && j < b.njobs; ++j) {
      const BatchJob &bj = b.jobs[j];
      int64_t *o = jobs + 7 * (int64_t)j;
      o[0] = bj.inst;
      o[1] = bj.parent;
      o[2] = bj.nchild;
      o[3] = bj.piv_row;
      o[4] = bj.row64;
      o[5] = bj.tile_begin;
      o[6] = bj.tile_count;
    }
  } catch (const std::bad_alloc &) {
    return fail(TSQR_ERR_OOM, "host allocation failed");
  }
  return TSQR_OK;
}

tsqr_status tsqr_factors_info(const tsqr_factors *F, int64_t *out) {
  if (!F || !out) return fail(TSQR_ERR_ARG, "NULL argument");
  if (!F->caqr()) {
    plan_info(F->plan(), out);
    return TSQR_OK;
  }
  // CAQR: totals over the panels (rows and columns of the whole matrix; the first
  // panel's tile rows and CTAs per SM)
  int64_t sum[8] = {0}, one[8];
  for (const tsqr_factors *P : F->panels) {
    plan_info(P->plan(), one);
    for (int i : {2, 4, 5, 6}) sum[i] += one[i];
  }
  plan_info(F->panels[0]->plan(), one);
  out[0] = F->mrows;
  out[1] = F->ncols;
  out[2] = sum[2];
  out[3] = one[3];
  out[4] = sum[4];
  out[5] = sum[5];
  out[6] = sum[6];
  out[7] = one[7];
  return TSQR_OK;
}

tsqr_status tsqr_profile_start(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (ProfRec &r : g_prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_prof.clear();
  g_prof_on = true;
  return TSQR_OK;
}

tsqr_status tsqr_profile_stop(int64_t max_records, int32_t *kind, float *ms, int64_t *count) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = false;
  tsqr_status st = TSQR_OK;
  const int64_t nrec = (int64_t)g_prof.size();
  if (count) *count = nrec;
  for (int64_t i = 0; i < nrec; ++i) {
    ProfRec &r = g_prof[i];
    if (i < max_records && kind && ms) {
      float t = 0.f;
      cudaError_t e = cudaEventSynchronize(r.b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
      if (e != cudaSuccess) st = fail(TSQR_ERR_CUDA, "profile readback: %s", cudaGetErrorString(e));
      kind[i] = r.kind;
      ms[i] = t;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_prof.clear();
  return st;
}

}  // extern "C"
