// Device code of one refinement task of the mixed-precision least-squares path, shared by
// the per-step launches (refine_batch.cu) and the resident kernel (resident.cu). The
// method and the task layout are described in refine_batch.cu.
#pragma once
#include <cstdint>

#include "tsqr_internal.h"

namespace tsqr {
namespace {

constexpr int kRThreads = 256;

__device__ __forceinline__ int refine_rc(int n) { return n <= 32 ? 256 : (n <= 64 ? 128 : 64); }

// the last arriver's solve: R (upper, FP64, ld ldr) staged packed; y holds g on entry,
// d on exit (layout y[c * K + j]); one warp
template <int K>
__device__ void solve_normal(const RefineInst &in, double *Rp, double *y, int k, bool &singular) {
  const int n = in.n, lane = threadIdx.x & 31;
  singular = false;
  for (int i = 0; i < n; ++i) {  // R^T y = g: column i of R^T is row i of R
    const double rii = Rp[i * (i + 1) / 2 + i];
    if (rii == 0.0) singular = true;
    if (lane < k) y[i * K + lane] = (rii == 0.0) ? 0.0 : y[i * K + lane] / rii;
    __syncwarp();
    const int rem = n - i - 1;
    for (int e = lane; e < rem * k; e += 32) {
      const int l = i + 1 + e % rem, j = e / rem;
      y[l * K + j] = fma(-Rp[l * (l + 1) / 2 + i], y[i * K + j], y[l * K + j]);
    }
    __syncwarp();
  }
  for (int i = n - 1; i >= 0; --i) {  // R d = y
    const double rii = Rp[i * (i + 1) / 2 + i];
    if (lane < k) y[i * K + lane] = (rii == 0.0) ? 0.0 : y[i * K + lane] / rii;
    __syncwarp();
    for (int e = lane; e < i * k; e += 32) {
      const int l = e % i, j = e / i;
      y[l * K + j] = fma(-Rp[i * (i + 1) / 2 + l], y[i * K + j], y[l * K + j]);
    }
    __syncwarp();
  }
}

// COH: A, B and the step history are read through L2 only (the resident kernel, whose
// inputs and tables change while it runs). decision (shared memory, two words, required
// with COH, else optional): the last task of the step writes 1 (refine on) or 2 (stopped)
// to decision[0]; the other tasks leave it alone.
template <int K, int T, bool COH = false>
__device__ void refine_task(const RefineParams &p, const RefineTask &tk, const RefineInst &in,
                            unsigned char *smraw, int *decision = nullptr) {
  double *sm = reinterpret_cast<double *>(smraw);
  const int n = in.n, k = in.k, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int RC = refine_rc(n), RCp = RC + 1, Q = kRThreads / RC;
  double *xs = sm;                        // n * K
  double *rs = xs + n * K;                // RC * K
  double *red = rs + RC * K;              // 256 * K
  double *As = red + kRThreads * K;       // max(RCp * n, 8 * S * n * K)
  const int NL = n >= 32 ? 32 : n;
  const int S = 32 / NL;
  const int tc = (n + 31) / 32;
  const int sub = lane / NL, cl = lane % NL;
  const bool lane_ok = sub < S;
  const bool first = p.step == 0;

  for (int e = tid; e < n * K; e += kRThreads) {
    const int c = e / K, j = e % K;
    xs[e] = (!first && j < k) ? __ldcg(in.X + c + (int64_t)j * in.ldx) : 0.0;
  }
  double acc2[T][K];
#pragma unroll
  for (int t = 0; t < T; ++t)
#pragma unroll
    for (int j = 0; j < K; ++j) acc2[t][j] = 0.0;

  for (int64_t r0 = tk.row0; r0 < tk.row0 + tk.rows; r0 += RC) {
    const int64_t left = tk.row0 + tk.rows - r0;
    const int rc = left < RC ? (int)left : RC;
    // stage the chunk (zero rows past its end)
    for (int c = w; c < n; c += kRThreads / 32) {
      const double *src = in.A + r0 + (int64_t)c * in.lda;
      for (int i = lane; i < RC; i += 32) As[c * RCp + i] = (i < rc) ? ld_input<COH>(src + i) : 0.0;
    }
    __syncthreads();
    // residual: thread (row i, column class q) sums over c = q, q + Q, ...
    {
      const int i = tid % RC, q = tid / RC;
      double acc[K];
#pragma unroll
      for (int j = 0; j < K; ++j) acc[j] = 0.0;
      if (!first) {
        for (int c = q; c < n; c += Q) {
          const double a = As[c * RCp + i];
#pragma unroll
          for (int j = 0; j < K; ++j) acc[j] = fma(a, xs[c * K + j], acc[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < K; ++j) red[(q * RC + i) * K + j] = acc[j];
    }
    __syncthreads();
    for (int e = tid; e < RC * K; e += kRThreads) {
      const int i = e % RC, j = e / RC;
      double v = 0.0;
      if (i < rc && j < k) {
        double s = 0.0;
        for (int q = 0; q < Q; ++q) s += red[(q * RC + i) * K + j];
        v = ld_input<COH>(in.B + r0 + i + (int64_t)j * in.ldb) - s;
      }
      rs[i * K + j] = v;
    }
    __syncthreads();
    // A^T r: lanes over columns (and row groups when n < 32), warps over rows
    if (lane_ok) {
      for (int i = w * S + sub; i < rc; i += 8 * S) {
        double rv[K];
#pragma unroll
        for (int j = 0; j < K; ++j) rv[j] = rs[i * K + j];
#pragma unroll
        for (int t = 0; t < T; ++t) {
          const int c = t * 32 + cl;
          if (t < tc && c < n) {
            const double a = As[c * RCp + i];
#pragma unroll
            for (int j = 0; j < K; ++j) acc2[t][j] = fma(a, rv[j], acc2[t][j]);
          }
        }
      }
    }
    __syncthreads();
  }

  // the task's partial g = sum over warps and row groups, in a fixed order
  double *wp = As;
  if (lane_ok) {
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const int c = t * 32 + cl;
      if (t < tc && c < n)
#pragma unroll
        for (int j = 0; j < K; ++j) wp[((w * S + sub) * n + c) * K + j] = acc2[t][j];
    }
  }
  __syncthreads();
  double *Pt = in.P + (int64_t)tk.idx * n * k;
  for (int e = tid; e < n * k; e += kRThreads) {
    const int c = e % n, j = e / n;
    double s = 0.0;
    for (int u = 0; u < 8 * S; ++u) s += wp[(u * n + c) * K + j];
    Pt[c + j * n] = s;
  }

  // arrive; the last task of the item finishes the step
  // the arrival flag: a word of the caller's shared memory in the resident kernel (its
  // static shared memory stays within the batch planner's slack), else this function's own
  int *last;
  if constexpr (COH) {
    last = decision + 1;
  } else {
    __shared__ int s_last;
    last = &s_last;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) *last = (atomicAdd(in.counter, 1) == in.nt - 1);
  __syncthreads();
  if (!*last) return;
  __threadfence();

  double *Rp = sm;                         // packed upper triangle, n (n + 1) / 2
  double *y = Rp + n * (n + 1) / 2;        // n * K
  for (int e = tid; e < n * n; e += kRThreads) {
    const int l = e % n, i = e / n;
    if (l <= i) Rp[i * (i + 1) / 2 + l] = __ldcg(in.R + l + (int64_t)i * in.ldr);
  }
  for (int e = tid; e < n * K; e += kRThreads) {
    const int c = e / K, j = e % K;
    double s = 0.0;
    if (j < k)
      for (int t = 0; t < in.nt; ++t) s += __ldcg(in.P + (int64_t)t * n * k + c + j * n);
    y[e] = s;
  }
  __syncthreads();
  if (w != 0) return;
  bool singular;
  solve_normal<K>(in, Rp, y, k, singular);
  double dn = 0.0, xn = 0.0;
  if (!singular) {
    for (int e = lane; e < n * k; e += 32) {
      const int c = e % n, j = e / n;
      double *xp = in.X + c + (int64_t)j * in.ldx;
      const double d = y[c * K + j];
      const double xv = first ? d : __ldcg(xp) + d;
      *xp = xv;
      dn = fma(d, d, dn);
      xn = fma(xv, xv, xn);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dn += __shfl_xor_sync(0xffffffffu, dn, o);
    xn += __shfl_xor_sync(0xffffffffu, xn, o);
  }
  if (lane == 0) {
    bool stop = (p.step == p.max_steps - 1);
    double ratio = 0.0;
    if (singular) {
      atomicExch(in.status, (int)TSQR_ERR_SINGULAR);
      stop = true;
    } else {
      ratio = (xn > 0.0) ? sqrt(dn / xn) : (dn > 0.0 ? 1.0 : 0.0);
      if (ratio <= 1e-15) stop = true;
      if (p.step >= 1) {
        // the contraction is not constant from step to step, so the prediction takes the
        // largest ratio of successive corrections seen so far
        const double prev = ld_state<COH>(in.hist + p.step - 1);
        double rho = 0.0;
        for (int s = 1; s <= p.step; ++s) {
          const double a = (s == p.step) ? ratio : ld_state<COH>(in.hist + s), b = ld_state<COH>(in.hist + s - 1);
          if (b > 0.0) rho = fmax(rho, a / b);
        }
        if (p.step >= 2 && ratio > 0.5 * prev) {
          stop = true;  // no more contraction: the rounding level is reached
        } else if (rho < 0.5 && ratio * rho / (1.0 - rho) <= p.tol) {
          stop = true;  // the predicted remaining error is below tol
        }
      }
    }
    in.hist[p.step] = ratio;
    *in.counter = 0;
    if (stop) *in.done = 1;
    if (decision) *decision = stop ? 2 : 1;
  }
}

}  // namespace
}  // namespace tsqr
