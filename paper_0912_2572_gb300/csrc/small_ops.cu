// Small kernels around the TSQR path (sm_103a): sign normalisation of R (paper §2.2:
// the factorization is unique once diag(R) > 0), the sign scaling of Q^T B / Q B, the
// root block of the thin-Q formation, and the triangular solve of least squares.
#include "tsqr_internal.h"

namespace tsqr {
namespace {

// d_j = sign(R_jj) (sign(0) = +1); R_out = D * R (upper), zeros below the diagonal.
__global__ void k_extract_r(const double *__restrict__ V, int64_t ldv, int n, double *R, int64_t ldr,
                            double *d) {
  const int j = blockIdx.x;  // column
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double di = (V[i + (int64_t)i * ldv] < 0.0) ? -1.0 : 1.0;
    if (j == 0 && d) d[i] = di;
    if (R) R[i + (int64_t)j * ldr] = (i <= j) ? di * V[i + (int64_t)j * ldv] : 0.0;
  }
}

// rows 0..n-1 of B (k columns) <- D * rows
__global__ void k_scale_rows(double *B, int64_t ldb, int n, int k, const double *__restrict__ d) {
  const int c = blockIdx.x;
  if (c >= k) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x) B[i + (int64_t)c * ldb] *= d[i];
}

// rows 0..n-1 of Q <- diag(d) (the root block of Q [I_n; 0] with the sign convention)
__global__ void k_formq_init(double *Q, int64_t ldq, int n, const double *__restrict__ d) {
  const int j = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) Q[i + (int64_t)j * ldq] = (i == j) ? d[j] : 0.0;
}

// X(:, c) = R^{-1} C(:, c) by back substitution, one CTA per right-hand side. R is the
// upper triangle of an n-by-n block (n <= 1024). A zero pivot sets *status = 4.
__global__ void k_trsv(const double *__restrict__ R, int64_t ldr, int n, const double *__restrict__ C,
                       int64_t ldc, double *X, int64_t ldx, const double *__restrict__ d, int32_t *status) {
  extern __shared__ double xs[];
  const int c = blockIdx.x;
  // with D = diag(d): (D R)^{-1} C = R^{-1} (D C), D = D^{-1}
  for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = d ? d[i] * C[i + (int64_t)c * ldc] : C[i + (int64_t)c * ldc];
  __syncthreads();
  __shared__ double xi_s;
  for (int i = n - 1; i >= 0; --i) {
    if (threadIdx.x == 0) {
      const double rii = R[i + (int64_t)i * ldr];
      if (rii == 0.0) {
        if (status) atomicExch(status, 4);
        xi_s = 0.0;
      } else {
        xi_s = xs[i] / rii;
      }
      xs[i] = xi_s;
    }
    __syncthreads();
    const double xi = xi_s;
    for (int t = threadIdx.x; t < i; t += blockDim.x) xs[t] = fma(-R[t + (int64_t)i * ldr], xi, xs[t]);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) X[i + (int64_t)c * ldx] = xs[i];
}

// FP64 FMA throughput probe (the roofline denominator of the FP64 kernels): every thread
// runs kProbeChains independent DFMA chains, enough to keep the FP64 pipe issuing.
// Thread 0 of block 0 also records the SM cycles and nanoseconds it ran (clk[0], clk[1]).
constexpr int kProbeChains = 8;
__device__ __forceinline__ uint64_t probe_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__global__ void k_dfma_probe(double *out, int iters, double a, double b, unsigned long long *clk) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  double x[kProbeChains];
#pragma unroll
  for (int u = 0; u < kProbeChains; ++u) x[u] = gid * 1e-12 + u;
  const uint64_t c0 = clock64(), t0 = probe_ns();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kProbeChains; ++u) x[u] = fma(x[u], a, b);
  }
  const uint64_t c1 = clock64(), t1 = probe_ns();
  if (gid == 0) {
    clk[0] = c1 - c0;
    clk[1] = t1 - t0;
  }
  double sum = 0.0;
#pragma unroll
  for (int u = 0; u < kProbeChains; ++u) sum += x[u];
  out[gid] = sum;
}

// FP64 tensor-core (DMMA) throughput probe: every warp runs kDmmaChains independent
// accumulator chains of mma.sync m8n8k4 FP64 (256 FMAs per warp instruction), operands
// from runtime values. Thread 0 of block 0 records cycles and nanoseconds as above.
constexpr int kDmmaChains = 4;
__global__ void k_dmma_probe(double *out, int iters, double a, double b, unsigned long long *clk) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[kDmmaChains][2];
#pragma unroll
  for (int u = 0; u < kDmmaChains; ++u) {
    acc[u][0] = gid * 1e-12 + u;
    acc[u][1] = gid * 1e-12 - u;
  }
  const double fa = a + gid * 1e-15, fb = b - gid * 1e-15;
  const uint64_t c0 = clock64(), t0 = probe_ns();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kDmmaChains; ++u)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(acc[u][0]), "+d"(acc[u][1])
                   : "d"(fa), "d"(fb));
  }
  const uint64_t c1 = clock64(), t1 = probe_ns();
  if (gid == 0) {
    clk[0] = c1 - c0;
    clk[1] = t1 - t0;
  }
  double sum = 0.0;
#pragma unroll
  for (int u = 0; u < kDmmaChains; ++u) sum += acc[u][0] + acc[u][1];
  out[gid] = sum;
}

}  // namespace

double launch_dmma_probe(double *out, unsigned long long *clk, int sms, int ctas_per_sm, int iters,
                         cudaStream_t s) {
  k_dmma_probe<<<sms * ctas_per_sm, 256, 0, s>>>(out, iters, 0.999999, 1e-7, clk);
  // 8 warps per CTA, each instruction 8 x 8 x 4 FMAs = 512 flops
  return 512.0 * kDmmaChains * (double)iters * 8.0 * sms * ctas_per_sm;
}

cudaError_t launch_extract_r(const double *V, int64_t ldv, int n, double *R, int64_t ldr, double *d,
                             cudaStream_t s) {
  k_extract_r<<<n, 128, 0, s>>>(V, ldv, n, R, ldr, d);
  return cudaGetLastError();
}

cudaError_t launch_scale_rows(double *B, int64_t ldb, int n, int k, const double *d, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_scale_rows<<<k, 128, 0, s>>>(B, ldb, n, k, d);
  return cudaGetLastError();
}

cudaError_t launch_formq_init(double *Q, int64_t ldq, int n, const double *d, cudaStream_t s) {
  k_formq_init<<<n, 128, 0, s>>>(Q, ldq, n, d);
  return cudaGetLastError();
}

cudaError_t launch_trsv(const double *R, int64_t ldr, int n, const double *C, int64_t ldc, int k,
                        double *X, int64_t ldx, const double *d, int32_t *status, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_trsv<<<k, 128, sizeof(double) * (size_t)n, s>>>(R, ldr, n, C, ldc, X, ldx, d, status);
  return cudaGetLastError();
}

// Launches the probe on a grid of SMs x ctas_per_sm CTAs of 256 threads; returns the
// flops it performs (2 per DFMA).
double launch_dfma_probe(double *out, unsigned long long *clk, int sms, int ctas_per_sm, int iters,
                         cudaStream_t s) {
  k_dfma_probe<<<sms * ctas_per_sm, 256, 0, s>>>(out, iters, 0.9999999, 1e-7, clk);
  return 2.0 * kProbeChains * (double)iters * 256.0 * sms * ctas_per_sm;
}

}  // namespace tsqr
