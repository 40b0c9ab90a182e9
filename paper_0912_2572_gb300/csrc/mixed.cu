// Kernels of the mixed-precision least-squares path (sm_103a).
//
// The leaves are factored in FP32 (the same TSQR kernel instantiated for float); the
// reduction tree over the leaves' triangles runs in FP64 on a compact array that holds
// only the chains' pivot blocks (chain c at rows c*n .. c*n+n-1). The solution is then
// refined in FP64 by Bjorck's augmented-system iterative refinement (Bjorck 1967;
// Higham, "Accuracy and Stability of Numerical Algorithms", §20.5): for the system
// [I A; A^T 0][r; x] = [b; 0] each step computes in FP64
//   f = b - r - A x,  g = -A^T r,
// solves for the correction with the mixed-precision QR,
//   [d1; d2] = Q^T f,  h = R^{-T} g,  dx = R^{-1} (d1 - h),  dr = Q [h; d2],
// and updates x += dx, r += dr in FP64. Starting from x = r = 0 the first step is the
// plain least-squares solve. The kernels here are the FP64 residual passes, the
// FP32 <-> FP64 hand-off of the pivot blocks, and the small per-step FP64 solve; every
// kernel of a step returns at once when the `done` flag says refinement has converged,
// so the host enqueues all steps without synchronizing.
#include <algorithm>

#include "tsqr_internal.h"

namespace tsqr {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// V64c rows [c*n, c*n+n) <- upper triangle of chain c's FP32 pivot block (its R).
__global__ void k_gather_r(const float *__restrict__ V32, int64_t ldv32, const int64_t *__restrict__ piv,
                           int n, double *__restrict__ V64, int64_t ldv64) {
  const int c = blockIdx.x;
  const int64_t pr = piv[c];
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    if (i <= j) V64[(int64_t)c * n + i + (int64_t)j * ldv64] = (double)V32[pr + i + (int64_t)j * ldv32];
  }
}

// B64c rows [c*n, c*n+n) <-> B32 pivot rows of chain c (k columns).
__global__ void k_gather_b(const float *__restrict__ B32, int64_t ldb32, const int64_t *__restrict__ piv,
                           int n, int k, double *__restrict__ B64, int64_t ldb64, const int32_t *done) {
  if (*done) return;
  const int c = blockIdx.x;
  const int64_t pr = piv[c];
  for (int e = threadIdx.x; e < n * k; e += blockDim.x) {
    const int i = e % n, col = e / n;
    B64[(int64_t)c * n + i + (int64_t)col * ldb64] = (double)B32[pr + i + (int64_t)col * ldb32];
  }
}

__global__ void k_scatter_b(float *__restrict__ B32, int64_t ldb32, const int64_t *__restrict__ piv, int n,
                            int k, const double *__restrict__ B64, int64_t ldb64, const int32_t *done) {
  if (*done) return;
  const int c = blockIdx.x;
  const int64_t pr = piv[c];
  for (int e = threadIdx.x; e < n * k; e += blockDim.x) {
    const int i = e % n, col = e / n;
    B32[pr + i + (int64_t)col * ldb32] = (float)B64[(int64_t)c * n + i + (int64_t)col * ldb64];
  }
}

// Per row i (one thread): r += dr (dr is the FP32 correction left in B32 by the
// previous step, skipped on the first step), then f = b - r - A x rounded into B32.
// x (n-by-k) is staged in shared memory.
template <int K>
__global__ void k_resid_f(const double *__restrict__ A, int64_t lda, int64_t m, int n, const double *__restrict__ b,
                          int64_t ldb, double *__restrict__ r, const double *__restrict__ x, float *__restrict__ B32,
                          int first, const int32_t *done) {
  if (*done) return;
  extern __shared__ double xs[];  // n * K
  for (int e = threadIdx.x; e < n * K; e += blockDim.x) xs[e] = x[e];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double f[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const double rc = first ? 0.0 : r[i + (int64_t)c * m] + (double)B32[i + (int64_t)c * m];
      r[i + (int64_t)c * m] = rc;
      f[c] = b[i + (int64_t)c * ldb] - rc;
    }
    for (int j = 0; j < n; ++j) {
      const double a = A[i + (int64_t)j * lda];
#pragma unroll
      for (int c = 0; c < K; ++c) f[c] = fma(-a, xs[j + c * n], f[c]);
    }
#pragma unroll
    for (int c = 0; c < K; ++c) B32[i + (int64_t)c * m] = (float)f[c];
  }
}

// g[j, c] -= sum_i A[i, j] r[i, c] over a chunk of rows: warp w of the CTA takes the
// columns j = w, w + 8, ..., lanes take rows; one warp reduction and an FP64 atomic add
// per output and CTA. g must be zero before the first chunk (the step kernel clears it).
template <int K>
__global__ void k_resid_g(const double *__restrict__ A, int64_t lda, int64_t m, int n, const double *__restrict__ r,
                          int64_t rows_per_cta, double *__restrict__ g, int first, const int32_t *done) {
  if (*done || first) return;  // r = 0 on the first step: g = 0
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t i0 = blockIdx.x * rows_per_cta;
  const int64_t i1 = min(m, i0 + rows_per_cta);
  for (int j = warp; j < n; j += nw) {
    double acc[K];
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = 0.0;
    for (int64_t i = i0 + lane; i < i1; i += 32) {
      const double a = A[i + (int64_t)j * lda];
#pragma unroll
      for (int c = 0; c < K; ++c) acc[c] = fma(a, r[i + (int64_t)c * m], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < K; ++c) {
      double v = acc[c];
#pragma unroll
      for (int s = 16; s >= 1; s >>= 1) v += __shfl_xor_sync(kFull, v, s);
      if (lane == 0) atomicAdd(&g[j + c * n], -v);
    }
  }
}

// One CTA: h = R^{-T} g, dx = R^{-1} (d1 - h), x += dx, root rows of B64c <- h, then
// hist[step] = ||dx||_F / ||x||_F and done = 1 when it is <= tol; g is cleared for the
// next step. R is the FP64 root triangle (raw signs, consistent with the raw Q^T).
// A zero pivot sets *status = 4 and stops the refinement.
__global__ void k_refine_step(const double *__restrict__ R, int64_t ldr, int n, int k, double *__restrict__ B64,
                              int64_t ldb64, double *__restrict__ g, double *__restrict__ x, double *__restrict__ hist,
                              int step, double tol, int32_t *done, int32_t *status) {
  if (*done) return;
  extern __shared__ double sm[];
  double *hs = sm;          // n * k : h
  double *ds = hs + n * k;  // n * k : d1 - h, then dx
  __shared__ double red[2];
  const int t = threadIdx.x;
  if (t < 2) red[t] = 0.0;
  for (int e = t; e < n * k; e += blockDim.x) hs[e] = g[e];
  __syncthreads();
  // forward substitution R^T h = g, column-oriented: for i: h_i /= r_ii; h_l -= r_il h_i (l > i)
  for (int i = 0; i < n; ++i) {
    for (int c = t; c < k; c += blockDim.x) {
      const double rii = R[i + (int64_t)i * ldr];
      if (rii == 0.0) {
        atomicExch(status, 4);
        hs[i + c * n] = 0.0;
      } else {
        hs[i + c * n] /= rii;
      }
    }
    __syncthreads();
    for (int e = t; e < (n - i - 1) * k; e += blockDim.x) {
      const int l = i + 1 + e % (n - i - 1), c = e / (n - i - 1);
      hs[l + c * n] = fma(-R[i + (int64_t)l * ldr], hs[i + c * n], hs[l + c * n]);
    }
    __syncthreads();
  }
  for (int e = t; e < n * k; e += blockDim.x) {
    const int i = e % n, c = e / n;
    ds[e] = B64[i + (int64_t)c * ldb64] - hs[e];
    B64[i + (int64_t)c * ldb64] = hs[e];
    g[e] = 0.0;
  }
  __syncthreads();
  // back substitution R dx = d1 - h
  for (int i = n - 1; i >= 0; --i) {
    for (int c = t; c < k; c += blockDim.x) {
      const double rii = R[i + (int64_t)i * ldr];
      ds[i + c * n] = (rii == 0.0) ? 0.0 : ds[i + c * n] / rii;
    }
    __syncthreads();
    for (int e = t; e < i * k; e += blockDim.x) {
      const int l = e % i, c = e / i;
      ds[l + c * n] = fma(-R[l + (int64_t)i * ldr], ds[i + c * n], ds[l + c * n]);
    }
    __syncthreads();
  }
  double sdx = 0.0, sx = 0.0;
  for (int e = t; e < n * k; e += blockDim.x) {
    const int i = e % n, c = e / n;
    const double nx = x[i + c * n] + ds[e];
    x[i + c * n] = nx;
    sdx = fma(ds[e], ds[e], sdx);
    sx = fma(nx, nx, sx);
  }
  atomicAdd(&red[0], sdx);
  atomicAdd(&red[1], sx);
  __syncthreads();
  if (t == 0) {
    const double rel = red[1] > 0.0 ? sqrt(red[0] / red[1]) : sqrt(red[0]);
    if (hist) hist[step] = rel;
    if (rel <= tol || *status != 0) *done = 1;
  }
}

}  // namespace

cudaError_t launch_gather_r(const float *V32, int64_t ldv32, const int64_t *piv, int G, int n, double *V64,
                            int64_t ldv64, cudaStream_t s) {
  k_gather_r<<<G, 256, 0, s>>>(V32, ldv32, piv, n, V64, ldv64);
  return cudaGetLastError();
}

cudaError_t launch_gather_b(const float *B32, int64_t ldb32, const int64_t *piv, int G, int n, int k, double *B64,
                            int64_t ldb64, const int32_t *done, cudaStream_t s) {
  k_gather_b<<<G, 128, 0, s>>>(B32, ldb32, piv, n, k, B64, ldb64, done);
  return cudaGetLastError();
}

cudaError_t launch_scatter_b(float *B32, int64_t ldb32, const int64_t *piv, int G, int n, int k, const double *B64,
                             int64_t ldb64, const int32_t *done, cudaStream_t s) {
  k_scatter_b<<<G, 128, 0, s>>>(B32, ldb32, piv, n, k, B64, ldb64, done);
  return cudaGetLastError();
}

cudaError_t launch_resid(const double *A, int64_t lda, int64_t m, int n, int k, const double *b, int64_t ldb,
                         double *r, const double *x, float *B32, double *g, int first, const int32_t *done,
                         int sms, cudaStream_t s) {
  const int threads = 256;
  const int64_t blocks_f = std::min<int64_t>((m + threads - 1) / threads, (int64_t)sms * 16);
  const size_t sm_f = sizeof(double) * (size_t)n * k;
  const int64_t rows_g = std::max<int64_t>(4096, (m + (int64_t)sms * 8 - 1) / ((int64_t)sms * 8));
  const int64_t blocks_g = (m + rows_g - 1) / rows_g;
#define TSQR_RESID(K)                                                                              \
  case K:                                                                                          \
    k_resid_f<K><<<(unsigned)blocks_f, threads, sm_f, s>>>(A, lda, m, n, b, ldb, r, x, B32, first, done); \
    k_resid_g<K><<<(unsigned)blocks_g, threads, 0, s>>>(A, lda, m, n, r, rows_g, g, first, done);  \
    break;
  switch (k) {
    TSQR_RESID(1)
    TSQR_RESID(2)
    TSQR_RESID(3)
    TSQR_RESID(4)
    TSQR_RESID(5)
    TSQR_RESID(6)
    TSQR_RESID(7)
    TSQR_RESID(8)
    default:
      return cudaErrorInvalidValue;
  }
#undef TSQR_RESID
  return cudaGetLastError();
}

cudaError_t launch_refine_step(const double *R, int64_t ldr, int n, int k, double *B64, int64_t ldb64, double *g,
                               double *x, double *hist, int step, double tol, int32_t *done, int32_t *status,
                               cudaStream_t s) {
  k_refine_step<<<1, 256, sizeof(double) * 2 * (size_t)n * k, s>>>(R, ldr, n, k, B64, ldb64, g, x, hist, step, tol,
                                                                    done, status);
  return cudaGetLastError();
}

}  // namespace tsqr
