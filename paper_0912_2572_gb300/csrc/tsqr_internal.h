// Internal declarations shared by the TSQR host code and kernels (not part of the C ABI).
//
// Execution model. A factorization is a list of launches; each launch runs a list of
// independent jobs, one CTA per job. A job owns a block of n "pivot rows" (the rows that
// end up holding its R) and walks a sequence of tiles:
//   GEQRT  dense Householder QR of a leaf's first tile; the pivot rows are the tile's own
//          first n rows (paper §2.2, a domain factorization);
//   TSQRT  QR of [R; tile]: an upper triangle on top of a dense tile (the flat-tree step
//          of paper §2.3, triangle-on-square);
//   TTQRT  QR of [R; R_child]: two stacked triangles (the binary reduce operator of
//          paper §2.3).
// A chain job = GEQRT + TSQRT...: a leaf taller than one tile, or a flat tree over
// leaves. A combine job = TTQRT...: one node of the reduction tree (k-1 children folded
// into the first child's rows). Reflector j of every tile has the form
// v = [1 at pivot row j; scale_j * (tile column j on its tail rows)], H = I - tau_j v v^T.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/tsqr.h"

namespace tsqr {

enum TileKind : int32_t { GEQRT = 0, TSQRT = 1, TTQRT = 2 };

struct TileDesc {
  int64_t row0;   // first global row of the tile
  int64_t refl;   // index of reflector 0 of this tile in the tau/scale arrays
  int32_t nrows;  // rows in the tile (TTQRT: n, or a piece of the child's triangle)
  int32_t kind;   // TileKind
  int32_t off;    // TTQRT piece: the tile's row 0 is row `off` of the child's triangle
  int32_t pad;
};

#ifdef __CUDACC__
template <bool COH>
__device__ __forceinline__ TileDesc load_tile(const TileDesc *t) {
  if constexpr (COH) {
    static_assert(sizeof(TileDesc) == 32, "four 8-byte loads");
    const long long *q = reinterpret_cast<const long long *>(t);
    const int2 a = __ldcg(reinterpret_cast<const int2 *>(q + 2)), b = __ldcg(reinterpret_cast<const int2 *>(q + 3));
    TileDesc d;
    d.row0 = __ldcg(q);
    d.refl = __ldcg(q + 1);
    d.nrows = a.x;
    d.kind = a.y;
    d.off = b.x;
    d.pad = b.y;
    return d;
  } else {
    return *t;
  }
}
#endif

struct JobDesc {
  int64_t piv_row;     // first of the n pivot rows
  int32_t tile_begin;  // index into the tile array
  int32_t tile_count;
};

struct LaunchDesc {
  int32_t job_begin;
  int32_t job_count;
};

// Tail rows [lo, hi) of reflector j within a tile of `ht` rows (empty when hi <= lo).
// A TTQRT tile holds rows off..off+ht-1 of the child's triangle, whose column j is
// nonzero on rows 0..j only.
__host__ __device__ inline void refl_rows(int kind, int j, int ht, int &lo, int &hi, int off = 0) {
  if (kind == GEQRT) {
    lo = j + 1;
    hi = ht;
  } else if (kind == TSQRT) {
    lo = 0;
    hi = ht;
  } else {
    lo = 0;
    hi = j + 1 - off;
    if (hi > ht) hi = ht;
    if (hi < 0) hi = 0;
  }
}

// Loads of kernel inputs. The launch-per-call kernels read their inputs through the
// read-only cache (COH = false); the resident kernel runs while the host replaces inputs
// and tables at reused addresses, so it reads them through L2 only (COH = true), where
// another SM's stale L1 line cannot be hit.
#ifdef __CUDACC__
template <bool COH>
__device__ __forceinline__ double ld_input(const double *p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}
template <bool COH>
__device__ __forceinline__ double2 ld_input(const double2 *p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}
// State another CTA of the same launch writes (COH) or written before the launch.
template <bool COH>
__device__ __forceinline__ double ld_state(const double *p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}
#endif

// ----------------------------------------------------------------- factor kernel
// R is the element type of the factorization (double; float for the leaves of the
// mixed-precision path). The input A is always FP64 and is rounded on load.
// Index checks of a build compiled with -DTSQR_CHECK (libtsqr_check.so): a job or tile
// descriptor that would take a kernel outside its buffers sets kErrBounds in the device
// error word (params `err`) and the job is skipped; nothing traps. A bound of 0 is
// unchecked. Normal builds compile the checks away.
#ifdef TSQR_CHECK
#define TSQR_CHECK_OR_SKIP(cond, err)         \
  if (!(cond)) {                              \
    if ((err) != nullptr) atomicOr((err), 2); \
    return;                                   \
  }
#else
#define TSQR_CHECK_OR_SKIP(cond, err)
#endif

template <typename R>
struct FactorParamsT {
  const double *A;  // first-touch input for GEQRT/TSQRT tiles
  int64_t lda;
  R *V;             // reflector and R storage, m-by-n
  int64_t ldv;
  R *B;             // optional extra columns (Q^T B fused), m-by-(nc-n), in place
  int64_t ldb;
  const JobDesc *jobs;
  const TileDesc *tiles;
  R *tau;
  R *scl;
  int32_t n;
  int32_t nc;   // n + extra columns
  int32_t ldt;  // tile capacity in rows (shared-memory leading dimension)
  int32_t job0; // first job of this launch
  // bounds for TSQR_CHECK builds (0 = unchecked): rows of V / A / B, entries of tau / scl,
  // descriptors; and the device error word
  int64_t rows, nrefl;
  int32_t ntiles, njobs;
  int32_t *err;
};
using FactorParams = FactorParamsT<double>;

// FP32 chains keep their tile in registers: kF32Rpt rows per lane, 16 lanes per column.
constexpr int kF32Rpt = 8;
constexpr int kF32TileRows = 16 * kF32Rpt;

// Shared memory of a factor job: the tile plus its step buffers (FP64), or only the
// step buffers of a register-tile FP32 chain (elem = 4).
size_t factor_smem_bytes(int nc, int ldt, size_t elem = sizeof(double));
// extra shared memory of an FP32 chain job with compact-WY panels (V twice, a chunk of
// trailing columns, V^T C, T^T W, G and T)
size_t f32wy_smem_extra_bytes();
// ctas_per_sm: CTAs per SM the tile height was planned for (3 selects the build that fits
// three in the register file; anything else, two).
cudaError_t launch_factor(const FactorParamsT<double> &p, int njobs, cudaStream_t s, int ctas_per_sm = 2);
int factor_max_rows(int nc, int ctas_per_sm, size_t smem_per_sm, size_t reserved_per_block,
                    size_t optin_per_block, size_t elem = sizeof(double));
// Tile height and CTAs per SM of an FP64 factorization (nc columns, n of them A's, leaves
// of leaf_h rows): three CTAs per SM where their tile still holds 2n rows (more
// independent column steps in flight per SM), else two, else one; at most max_cps.
bool factor_tile_choice(int n, int nc, int leaf_h, size_t smem_per_sm, size_t reserved_per_block,
                        size_t optin_per_block, int max_cps, int &tile_h, int &cps);

// ---------------------------------------------------------- batched persistent kernel
// One launch factors every instance of a batch: CTAs take chain jobs from an atomic queue;
// when a job finishes, its CTA arrives at the parent tree node (an atomic counter) and
// the last child to arrive runs the node's combine, then climbs on. No CTA ever waits.
// The CTA that completes an instance's root writes R (diag >= 0) and, with right-hand
// sides fused into the factorization, solves R X = (Q^T B)[0:n].
struct BatchInst {
  const double *A;  // input, m-by-n, leading dimension lda
  int64_t lda;
  void *V;          // chain storage: double (FP64) or float (mixed), m-by-n, ld = ldv
  int64_t ldv;
  double *B;        // fused right-hand sides (library copy, m-by-k) or null
  int64_t ldb;
  void *tau, *scl;  // chain reflector scalars (same element type as V)
  double *V64;      // tree storage: V itself (FP64) or the compact pivot blocks (mixed)
  int64_t ldv64;
  double *tau64, *scl64;
  double *R;        // optional output, n-by-n
  int64_t ldr;
  double *X;        // optional output, n-by-k
  int64_t ldx;
  int32_t *status;  // device flag set to 4 when R is singular (solve only)
  int32_t n, k, ldt, mixed;
  int32_t ldt_tree;  // shared-memory rows of a tree-node tile (a piece of a triangle)
  int32_t wy;        // mixed items: FP32 chains by compact-WY panels with 3xTF32 tensor-core
                     // updates (run_job_f32wy) instead of the unblocked register tile
};

struct BatchJob {   // chain jobs first (queue order), then tree nodes
  int64_t piv_row;  // pivot rows in the job's storage (V for chains, V64 for nodes)
  int64_t row64;    // where the job's triangle lives in the tree storage
  int32_t tile_begin, tile_count;
  int32_t inst, parent;  // parent node (job index) or -1 at the root
  int32_t nchild, pad;   // arrivals a node waits for (its children)
};

struct BatchParams {
  const BatchInst *inst;
  const BatchJob *jobs;
  const TileDesc *tiles;
  int32_t *counters;  // one per job, zero at launch
  int32_t *queue;     // next chain job, zero at launch
  int32_t nchains;
};

cudaError_t launch_factor_batch(const BatchParams &p, int cmax, int grid, size_t smem_bytes, cudaStream_t s,
                                bool wy = false);

// ------------------------------------------------------- cluster tier of the tree
// With TSQR_CLUSTER, three binary tree levels run in one launch of thread-block clusters
// of kClusterSize CTAs: cluster c reduces the 8 consecutive triangles 8c..8c+7 of the
// level below (4 + 2 + 1 combine jobs, one CTA each). A combine's column step j needs only
// row j of each child's output triangle, which is final once the child has finished its
// own step j, so the levels run as a pipeline: a parent waits for its children's progress
// counters and reads their rows from their shared memory (distributed shared memory).
constexpr int kClusterSize = 8;
struct ClusterSlot {
  int32_t job;       // combine job of this CTA, or -1 (idle)
  int32_t child[2];  // cluster rank producing the pivot (0) / tile (1) triangle, or -1 when
                     // that triangle is complete in global memory (an earlier launch's)
  int32_t pad;
};
// Shared memory of a cluster-tier combine CTA (the child's triangle, the dot products and
// the pivot triangle), 0 when it exceeds the per-block maximum.
size_t cluster_smem_bytes(int n, int nc, size_t optin_per_block);
// err: the device error word (bit kErrTimeout set when a bounded wait gave up).
cudaError_t launch_factor_cluster(const FactorParamsT<double> &p, const ClusterSlot *slots, int nclusters,
                                  int32_t *err, cudaStream_t s);

// Device error word: bit 1 (kErrTimeout) a bounded device wait gave up, bit 2 (kErrBounds)
// an index check of a TSQR_CHECK build failed. One word per device.
constexpr int32_t kErrTimeout = 1;
constexpr int32_t kErrBounds = 2;
cudaError_t device_error_word(int32_t **ptr);  // the current device's word

// ------------------------------------------------ batched least-squares refinement
// Mixed-precision least-squares items of a batch: after the batched factorization, one
// launch per step of corrected semi-normal-equation refinement (refine_batch.cu). A
// refinement instance is one item and a group of at most 8 right-hand sides.
struct RefineInst {
  const double *A;     // the item's A, m-by-n, lda
  int64_t lda;
  const double *B;     // the group's right-hand sides, m-by-k, ldb
  int64_t ldb;
  double *X;           // the group's solution columns, n-by-k, ldx (written from step 0)
  int64_t ldx;
  const double *R;     // the item's FP64 R (upper triangle; any diagonal signs), ldr
  int64_t ldr;
  double *P;           // partial A^T r of each task, nt blocks of n-by-k
  int32_t *counter;    // task arrivals of the current step (reset by the last one)
  int32_t *done;       // 1 once the group has converged or R is singular
  int32_t *status;     // the item's status word (TSQR_ERR_SINGULAR)
  double *hist;        // ||dX||_F / ||X||_F per step
  int32_t n, k, kb, nt;  // kb = the kernel's register width for k (k itself); nt = tasks
};

struct RefineTask {
  int64_t row0;        // first row of the task's block
  int32_t rows;
  int32_t inst;        // refinement instance
  int32_t idx;         // task index within the instance (partial slot)
  int32_t pad;
};

struct RefineParams {
  const RefineInst *inst;
  const RefineTask *tasks;
  int32_t step, max_steps;
  double tol;          // stop once the predicted remaining ||dX|| / ||X|| is below tol
};

int refine_rows_per_chunk(int n);
size_t refine_smem_bytes(int n, int kb);
cudaError_t launch_refine_batch(const RefineParams &p, int ntasks, size_t smem_bytes, cudaStream_t s);

// -------------------------------------------------------- resident persistent kernel
// The resident server keeps one persistent kernel on the GPU and admits requests into it
// while it runs (resident.cu, server.cu). The host appends each admitted request's chain
// jobs to a ring in device memory and then advances that ring's `tail`, both by copies on
// its upload stream (the copy of `tail` lands after the entries and tables it publishes).
// There are two host rings, one for requests of at most kResSmallChains chain jobs and one
// for larger ones; CTAs claim from the small ring first, so a short request does not wait
// behind the chain jobs of a long one. CTAs claim entries by compare-and-swap on `head`.
// Refinement tasks of mixed least-squares requests
// are produced on the device: the CTA that finishes a request's factorization (or a step
// of its refinement) reserves entries of a second ring (`dtail`), fills them and releases
// each with its sequence number. A CTA with nothing to claim polls (bounded); when it has
// seen no work for a while and no CTA is busy, it sets `quit` and the whole kernel ends;
// the host launches it again when work arrives. Completion is written to mapped host
// memory: the request's status, then its admission sequence number.
constexpr int kResSmallChains = 8;  // requests of at most this many chain jobs: ring 0

struct ResCtl {
  unsigned long long head[2], tail[2];  // host rings: next entry to claim, entries published
  unsigned long long dhead, dtail;  // device ring: next entry to claim, entries reserved
  int32_t busy;                     // CTAs running a claimed job
  int32_t quit;                     // set by a CTA to end the launch (reset by the host)
  int32_t stop;                     // set by the host: end once idle, without waiting
  int32_t pad;
};

struct ResEntry {  // host ring: chain job `job` of the request in slot `slot`
  int32_t slot, job;
};

struct ResTask {   // device ring: refinement task of (slot, group) for `step`
  int32_t slot, group, step, task;
  uint32_t seq;    // low 32 bits of (ring index + 1), written last
  int32_t pad[3];
};

struct ResItemDev {  // one admitted request, in the slot table (device memory)
  BatchInst inst;
  const BatchJob *jobs;
  const TileDesc *tiles;
  int32_t *counters;   // arrival counters of the request's jobs
  RefineInst *rinst;   // refinement groups (mixed least-squares requests)
  int32_t *pending;    // groups still refining
  int64_t m;
  int32_t nchains, ngroups, nt, seq;
};

struct ResParams {
  ResCtl *ctl;
  const ResEntry *ring;      // host ring c at ring + c * (ring_mask + 1), c = 0 (small), 1
  ResTask *dring;
  const ResItemDev *items;
  int32_t *hstatus, *hdone;  // mapped host memory, one word per slot
  int32_t *err;              // device error word
  unsigned long long ring_mask, dring_mask;  // capacities - 1 (powers of two)
  int64_t idle_polls;        // consecutive empty polls before a CTA tries to end the launch
  int64_t refine_rows;       // rows per refinement task
  int32_t max_steps;
  double tol;
};

cudaError_t launch_resident(const ResParams &p, int grid, size_t smem_bytes, cudaStream_t s);

// One request planned for the resident kernel (host side, tsqr_api.cu): the batched
// planner's tables for this one item and the size of its device block.
struct ResidentPlan {
  size_t bytes = 0;  // device block (workspaces, tables, counters)
  size_t smem = 0;   // shared memory its jobs need
  int cmax = 1;
  int32_t nchains = 0, njobs = 0, ngroups = 0, nt = 0;
  bool wy = false;
  void *impl = nullptr;  // the planner's state (resident_plan_free)
};
tsqr_status resident_plan(const tsqr_batch_item &it, int32_t chain_tiles, ResidentPlan &out);
// Binds the plan to its device block at `base` and enqueues on s the uploads that make it
// runnable: tables, zeroed counters and status words, the library copy of B. Fills `dev`
// (its slot, seq and pending pointer set by the caller afterwards).
tsqr_status resident_upload(const ResidentPlan &p, char *base, cudaStream_t s, ResItemDev &dev);
void resident_plan_free(ResidentPlan &p);
// Dynamic shared memory of the resident kernel at `ctas_per_sm` CTAs per SM: the per-CTA
// budget of the batched planner (a request fits when its plan's smem is at most this).
size_t resident_smem_bytes(int ctas_per_sm);
int64_t refine_rows_per_task();
int32_t refine_max_steps();
double refine_tolerance();

// host side of the batched path (tsqr_api.cu), also driven by the server (server.cu)
tsqr_status batch_solve_internal(const tsqr_batch_item *items, int32_t count, int32_t chain_tiles, int32_t arity,
                                 cudaStream_t s, int32_t *status, int32_t *status_async, double *info,
                                 int32_t ctas_per_sm = 0);
tsqr_status check_batch_item(const tsqr_batch_item &it, int32_t q);
size_t batch_item_bytes(const tsqr_batch_item &it);  // device workspace estimate for admission
int32_t resolve_batch_prec(const tsqr_batch_item &it);  // TSQR_FP64 or TSQR_MIXED
const char *last_error_text();
size_t live_free_bytes();  // device memory free now, counting the pool's unused reserve
// failure injection (tsqr_debug_fail_allocations): true while injected failures remain,
// consuming one
bool debug_take_allocation_failure();
// the calling thread's error message (tsqr_last_error) for entry points outside tsqr_api.cu
tsqr_status set_last_error(tsqr_status s, const char *fmt, ...);
void clear_last_error();

// ------------------------------------------------------------------ apply kernels
template <typename R>
struct ApplyParamsT {
  const R *V;
  int64_t ldv;
  R *B;  // m-by-k target
  int64_t ldb;
  const JobDesc *jobs;
  const TileDesc *tiles;
  const R *tau;
  const R *scl;
  int32_t n;
  int32_t k;         // columns of B handled by this launch
  int32_t col0;      // first column of B (wide kernel passes)
  int32_t ldt;       // max tile rows
  int32_t job0;
  int32_t trans;     // 1: Q^T (forward order), 0: Q (reverse order)
  int32_t formq;     // 1: forming the thin Q (tiles start at zero, column j >= ref j only)
  // bounds for TSQR_CHECK builds (0 = unchecked), as FactorParamsT
  int64_t rows, nrefl;
  int32_t ntiles, njobs;
  int32_t *err;
};

using ApplyParams = ApplyParamsT<double>;

// cols_per_cta caps the columns of B one CTA of the tile kernel handles (16, 32 or 64): a
// launch with few jobs (a tree level) spreads a job's columns over more CTAs. Columns are
// independent; only the summation order of a column's dot products changes with the cap.
// tile_pairs: a launch whose jobs hold several tiles, with one column of B (Q^T b, Q b),
// runs the tile-pair kernel (the job's tiles alternate between the two half-warps).
cudaError_t launch_apply(const ApplyParamsT<double> &p, int njobs, cudaStream_t s, int ctas_per_sm = 2,
                         int cols_per_cta = 64, bool tile_pairs = false);

// Cluster tier of B <- Q B (top down): one CTA per combine of a cluster launch of the
// factorization's schedule, for 16 columns of B; parent = the cluster rank whose block this
// node's pivot rows come from (-1: complete in global memory), side 0 = the parent's pivot
// block, 1 = its tile block; kids bit q = the pivot (0) / tile (1) child is in the cluster.
struct ApplyClusterSlot {
  int32_t job;
  int32_t parent, side, kids;
};
size_t apply_cluster_smem_bytes(int n);
cudaError_t launch_apply_cluster(const ApplyParamsT<double> &p, const ApplyClusterSlot *slots, int nclusters,
                                 cudaStream_t s);

// ------------------------------------------------------------------- small kernels
cudaError_t launch_extract_r(const double *V, int64_t ldv, int n, double *R, int64_t ldr,
                             double *d, cudaStream_t s);
cudaError_t launch_scale_rows(double *B, int64_t ldb, int n, int k, const double *d,
                              cudaStream_t s);
cudaError_t launch_formq_init(double *Q, int64_t ldq, int n, const double *d, cudaStream_t s);

// The FP64 FMA throughput probe (out: one double per thread; clk: cycles and ns of one
// thread); returns the flops of one launch.
double launch_dfma_probe(double *out, unsigned long long *clk, int sms, int ctas_per_sm, int iters,
                         cudaStream_t s);
// The FP64 tensor-core (DMMA, mma.sync m8n8k4) throughput probe, same outputs.
double launch_dmma_probe(double *out, unsigned long long *clk, int sms, int ctas_per_sm, int iters,
                         cudaStream_t s);

// X = R^{-1} (D C[0:n]) for the raw upper triangle R (leading dimension ldr) and the
// optional sign vector d (NULL = no scaling); a zero pivot sets *status = 4.
cudaError_t launch_trsv(const double *R, int64_t ldr, int n, const double *C, int64_t ldc,
                        int k, double *X, int64_t ldx, const double *d, int32_t *status,
                        cudaStream_t s);

}  // namespace tsqr
