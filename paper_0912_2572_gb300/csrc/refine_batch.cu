// Batched least-squares refinement for the mixed-precision batched path (sm_103a).
//
// The paper computes R and Q in one precision and has no refinement step; this is the
// library's mixed-precision extension. The batched kernel factors each mixed item with
// FP32 leaf chains and an FP64 tree, giving an FP64 upper-triangular R that is the exact
// R factor of a matrix A + E with ||E|| of order u_32 ||A||. Each least-squares item is
// then solved by corrected semi-normal equations (Bjorck's CSNE, iterated): from x = 0,
//   r = b - A x,   g = A^T r   (both FP64, one pass over A),
//   R^T y = g,     R d = y,     x <- x + d.
// The iteration matrix I - R^{-1} R^{-T} A^T A has norm about 2 ||E R^{-1}|| ~ u_32 kappa,
// so each step gains about -log10(u_32 kappa) digits, down to the accuracy the FP64
// products allow (about u_64 kappa, plus u_64 kappa^2 ||r|| / (||A|| ||x||)). A group
// stops once its last correction times rho / (1 - rho) is below tol, rho the largest
// ratio of successive corrections so far, or once the corrections stop shrinking.
//
// One launch is one step for every item of the batch. A task is a block of rows of one
// item: its CTA stages the rows of A chunk by chunk in shared memory, computes r for the
// chunk (lanes over rows) and accumulates the chunk's A^T r (lanes over columns) in
// registers; at the end of the task it writes its partial g. The last task of an item to
// arrive (atomic counter) sums the partials in task order, so results do not depend on
// scheduling, and runs both triangular solves in one warp with R staged in shared memory.
// FP64 dominates the cost (4 m n k flops per step), so lanes are kept full: rows fill the
// lanes in the residual, columns (or columns x row groups when n < 32) in A^T r.
#include <algorithm>

#include "refine_task.cuh"
#include "tsqr_internal.h"

namespace tsqr {
namespace {

template <int K, int T>
__device__ __forceinline__ void refine_go(const RefineParams &p, const RefineTask &tk, const RefineInst &in,
                                          unsigned char *smraw) {
  refine_task<K, T>(p, tk, in, smraw);
}

__global__ void __launch_bounds__(kRThreads, 2) k_refine_batch(const RefineParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const RefineTask tk = p.tasks[blockIdx.x];
  const RefineInst in = p.inst[tk.inst];
  if (__ldcg(in.done) != 0) return;
  // exact right-hand-side count and column-tile count: a padded slot would still issue
  // its DFMA (a predicated-off lane occupies the FP64 pipe)
  const int tb = (in.n + 31) / 32;
#define TSQR_REFINE_CASE(K, T) \
  case K * 8 + T: refine_go<K, T>(p, tk, in, smraw); return;
#define TSQR_REFINE_K(K) \
  TSQR_REFINE_CASE(K, 1) TSQR_REFINE_CASE(K, 2) TSQR_REFINE_CASE(K, 3) TSQR_REFINE_CASE(K, 4)
  switch (in.kb * 8 + tb) {
    TSQR_REFINE_K(1) TSQR_REFINE_K(2) TSQR_REFINE_K(3) TSQR_REFINE_K(4)
    TSQR_REFINE_K(5) TSQR_REFINE_K(6) TSQR_REFINE_K(7) TSQR_REFINE_K(8)
    default: return;
  }
#undef TSQR_REFINE_K
#undef TSQR_REFINE_CASE
}

}  // namespace

int refine_rows_per_chunk(int n) { return n <= 32 ? 256 : (n <= 64 ? 128 : 64); }

size_t refine_smem_bytes(int n, int kb) {
  const int RC = refine_rows_per_chunk(n), RCp = RC + 1;
  const int NL = n >= 32 ? 32 : n, S = 32 / NL;
  const size_t as = std::max((size_t)RCp * n, (size_t)8 * S * n * kb);
  const size_t main = (size_t)n * kb + (size_t)RC * kb + (size_t)kRThreads * kb + as;
  const size_t solve = (size_t)n * (n + 1) / 2 + (size_t)n * kb;
  return sizeof(double) * std::max(main, solve);
}

cudaError_t launch_refine_batch(const RefineParams &p, int ntasks, size_t smem_bytes, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_refine_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e != cudaSuccess) return e;
  k_refine_batch<<<ntasks, kRThreads, smem_bytes, s>>>(p);
  return cudaGetLastError();
}

}  // namespace tsqr
