// tsqr_lstsq_static: FP64 least squares that allocates no memory.
//
// Some callers cannot allocate device memory: code running inside a host callback or a
// signal-safe section, plugins whose host framework owns every allocation, or
// applications that reserve the whole device up front and forbid later cudaMalloc /
// cudaMallocAsync calls. This entry point serves them: it runs the same FP64 path as
// tsqr_lstsq (TSQR of [A | B] with Q^T B fused into the factorization, two-level tree,
// then back substitution) but keeps all its scratch (reflector storage, the Q^T B
// workspace, the reflector scalars, the plan and a status word) in one file-scope
// device array of kStaticScratchBytes, and builds its plan in fixed host arrays. It calls
// no cudaMalloc, cudaFree or other allocating routine, and no heap allocation on the
// host.
//
// Costs and rules of use:
//   * every GPU that loads the library holds the array (64 MiB) until the process exits;
//   * the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current; the stream passed must belong to
//     the current device (checked);
//   * every call waits for its stream (it reads back the singularity flag), so no call,
//     the first included, can be made on a stream that is being captured into a graph;
//   * every call shares the one array, which keeps the previous call's contents: calls
//     that can overlap on the GPU (different streams, or several host threads) race on
//     it and must be serialized by the caller; host-side use is serialized by a mutex,
//     and a call that fails after enqueuing work waits for its stream before returning,
//     so that work never overlaps the next call;
//   * problems whose scratch exceeds the array, or whose plan exceeds the fixed host
//     arrays, are rejected with TSQR_ERR_UNSUPPORTED before any work is enqueued;
//   * errors are described by tsqr_last_error(), whose buffer is fixed (no allocation).
#include <mutex>

#include "../../include/tsqr.h"
#include "tsqr_internal.h"

using namespace tsqr;

namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
constexpr int kMaxTiles = 32768;
constexpr int kMaxJobs = 8192;
constexpr int kMaxLaunches = 64;

std::mutex g_mu;  // serializes the host-side plan arrays and the per-device set-up
void *g_dev_ptr[kMaxDevices];
TileDesc g_tiles[kMaxTiles];
JobDesc g_jobs[kMaxJobs];
LaunchDesc g_launches[kMaxLaunches];
int64_t g_piv[2][kMaxJobs];

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// The two-level tree of tsqr_factor (TSQR_TWO_LEVEL, arity 2) with leaves of one tile:
// chains of consecutive tiles inside a CTA, then a binary tree across chains.
bool build_plan(int64_t m, int n, int tile_h, int64_t chains_target, int &ntiles, int &njobs,
                int &nlaunches) {
  const int64_t P = m / tile_h > 0 ? m / tile_h : 1;
  const int64_t G = P < chains_target ? P : chains_target;
  if (G > kMaxJobs || P + G > kMaxTiles) return false;
  ntiles = njobs = nlaunches = 0;
  g_launches[nlaunches++] = {0, 0};
  for (int64_t c = 0; c < G; ++c) {
    const int64_t la = c * P / G, lb = (c + 1) * P / G;
    JobDesc job{la * tile_h, ntiles, 0};
    for (int64_t l = la; l < lb; ++l) {
      const int64_t r0 = l * tile_h, r1 = (l == P - 1) ? m : (l + 1) * tile_h;
      for (int64_t r = r0; r < r1; r += tile_h) {
        if (ntiles >= kMaxTiles) return false;
        const int64_t hh = (r1 - r < tile_h) ? r1 - r : tile_h;
        g_tiles[ntiles] = {r, (int64_t)ntiles * n, (int32_t)hh, ntiles == job.tile_begin ? GEQRT : TSQRT};
        ++ntiles;
      }
    }
    job.tile_count = ntiles - job.tile_begin;
    g_piv[0][njobs] = job.piv_row;
    g_jobs[njobs++] = job;
  }
  g_launches[0].job_count = njobs;
  int cur = 0;
  int64_t count = G;
  while (count > 1) {
    if (nlaunches >= kMaxLaunches) return false;
    LaunchDesc ld{njobs, 0};
    int64_t next = 0;
    for (int64_t g = 0; g < count; g += 2) {
      g_piv[cur ^ 1][next++] = g_piv[cur][g];
      if (g + 1 >= count) continue;
      if (njobs >= kMaxJobs || ntiles >= kMaxTiles) return false;
      g_jobs[njobs++] = {g_piv[cur][g], ntiles, 1};
      g_tiles[ntiles] = {g_piv[cur][g + 1], (int64_t)ntiles * n, n, TTQRT};
      ++ntiles;
    }
    ld.job_count = njobs - ld.job_begin;
    g_launches[nlaunches++] = ld;
    count = next;
    cur ^= 1;
  }
  return true;
}

}  // namespace

extern "C" tsqr_status tsqr_lstsq_static(const double *A, int64_t m, int32_t n, int64_t lda, const double *B,
                                         int64_t ldb, int32_t k, double *X, int64_t ldx, void *stream) {
  clear_last_error();
  if (!A || !B || !X) return set_last_error(TSQR_ERR_ARG, "A, B or X is NULL");
  if (n < 1 || k < 1 || n + k > 128) return set_last_error(TSQR_ERR_ARG, "n=%d, k=%d: need n, k >= 1 and n + k <= 128", n, k);
  if (m < n || lda < m || ldb < m || ldx < n)
    return set_last_error(TSQR_ERR_ARG, "bad sizes: m=%lld n=%d lda=%lld ldb=%lld ldx=%lld", (long long)m, n,
                          (long long)lda, (long long)ldb, (long long)ldx);
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_last_error(TSQR_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_last_error(TSQR_ERR_UNSUPPORTED, "device %d >= %d", dev, kMaxDevices);
  int sdev = dev;
  e = cudaStreamGetDevice(s, &sdev);
  if (e != cudaSuccess) return set_last_error(TSQR_ERR_CUDA, "cudaStreamGetDevice: %s", cudaGetErrorString(e));
  if (sdev != dev)
    return set_last_error(TSQR_ERR_ARG, "the stream belongs to device %d, the current device is %d", sdev, dev);
  if (!g_dev_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return set_last_error(TSQR_ERR_CUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
    g_dev_ptr[dev] = p;
  }
  int sms = 0, smem_sm = 0, reserved = 0, optin = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return set_last_error(TSQR_ERR_CUDA, "device %d attributes", dev);
  const int nc = n + k;
  int cps = 0, tile_h = 0;
  if (!factor_tile_choice(n, nc, 1 << 20, smem_sm, reserved, optin, 3, tile_h, cps))
    return set_last_error(TSQR_ERR_UNSUPPORTED, "no tile height fits shared memory for n + k = %d", nc);
  int ntiles = 0, njobs = 0, nlaunches = 0;
  if (!build_plan(m, n, tile_h, (int64_t)sms * cps * 4, ntiles, njobs, nlaunches))
    return set_last_error(TSQR_ERR_UNSUPPORTED, "m=%lld needs more than %d tiles or %d jobs", (long long)m, kMaxTiles,
                          kMaxJobs);
  // scratch layout inside the static array
  const size_t o_status = 0;
  const size_t o_jobs = o_status + 256;
  const size_t o_tiles = o_jobs + up256(sizeof(JobDesc) * njobs);
  const size_t o_tau = o_tiles + up256(sizeof(TileDesc) * ntiles);
  const size_t o_scl = o_tau + up256(sizeof(double) * ntiles * n);
  const size_t o_V = o_scl + up256(sizeof(double) * ntiles * n);
  const size_t o_W = o_V + up256(sizeof(double) * (size_t)m * n);
  const size_t need = o_W + up256(sizeof(double) * (size_t)m * k);
  if (need > kStaticScratchBytes)
    return set_last_error(TSQR_ERR_UNSUPPORTED, "scratch of %zu bytes exceeds the %zu-byte static array", need,
                          kStaticScratchBytes);
  char *base = (char *)g_dev_ptr[dev];
  int32_t *status = (int32_t *)(base + o_status);
  JobDesc *djobs = (JobDesc *)(base + o_jobs);
  TileDesc *dtiles = (TileDesc *)(base + o_tiles);
  double *tau = (double *)(base + o_tau), *scl = (double *)(base + o_scl);
  double *V = (double *)(base + o_V), *W = (double *)(base + o_W);

  // once work is enqueued, a failing step waits for the stream before returning, so that
  // nothing of this call still uses the shared array when the next call starts
#define STATIC_TRY(expr)                                                                \
  do {                                                                                  \
    const cudaError_t e_ = (expr);                                                      \
    if (e_ != cudaSuccess) {                                                            \
      cudaStreamSynchronize(s);                                                         \
      return set_last_error(TSQR_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_)); \
    }                                                                                   \
  } while (0)

  // the previous call's contents stay in the array: clear the status word, and copy
  // everything else in before it is read
  STATIC_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t), s));
  STATIC_TRY(cudaMemcpyAsync(djobs, g_jobs, sizeof(JobDesc) * njobs, cudaMemcpyHostToDevice, s));
  STATIC_TRY(cudaMemcpyAsync(dtiles, g_tiles, sizeof(TileDesc) * ntiles, cudaMemcpyHostToDevice, s));
  STATIC_TRY(cudaMemcpy2DAsync(W, sizeof(double) * m, B, sizeof(double) * ldb, sizeof(double) * m, k,
                               cudaMemcpyDeviceToDevice, s));
  FactorParams p{};
  p.A = A;
  p.lda = lda;
  p.V = V;
  p.ldv = m;
  p.B = W;
  p.ldb = m;
  p.jobs = djobs;
  p.tiles = dtiles;
  p.tau = tau;
  p.scl = scl;
  p.n = n;
  p.nc = nc;
  p.ldt = tile_h;
  for (int q = 0; q < nlaunches; ++q) {
    p.job0 = g_launches[q].job_begin;
    STATIC_TRY(launch_factor(p, g_launches[q].job_count, s, q == 0 ? cps : 2));
  }
  STATIC_TRY(launch_trsv(V, m, n, W, m, k, X, ldx, nullptr, status, s));
  int32_t hstatus = 0;
  STATIC_TRY(cudaMemcpyAsync(&hstatus, status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  STATIC_TRY(cudaStreamSynchronize(s));
#undef STATIC_TRY
  if (hstatus == 4) return set_last_error(TSQR_ERR_SINGULAR, "R has a zero diagonal entry");
  return TSQR_OK;
}
