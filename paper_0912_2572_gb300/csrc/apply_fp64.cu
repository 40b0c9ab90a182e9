// Application of the TSQR orthogonal factor (sm_103a): B <- Q^T B, B <- Q B, and the
// thin Q = Q [I_n; 0] (paper §4, Table 2: Q costs what R costs; Property 1).
//
// The factor set is a list of launches of jobs; each job walks its tiles and each tile
// holds n reflectors v = [1 at pivot row j; scale_j * tail_j] (tsqr_internal.h). Q^T
// applies jobs launch by launch, tiles and reflectors in factorization order; Q applies
// everything in reverse.
//
// Two kernels:
//   * k_apply_warp: one warp per job, for B with at most 8 columns. Each reflector is a
//     dot product over the tile rows, one warp-level transpose-reduce, and an update; no
//     block barrier is needed, so many jobs run per SM and hide the reduction latency.
//   * k_apply_wide: one CTA per job and per pass of 32 columns, the same half-warp
//     column mapping as the factor kernel. Used for many right-hand sides and for
//     forming Q. When forming Q every pivot-row block stays upper triangular (the
//     root starts from diag(sign(r_jj)) and each node's Q blocks are triangular), so
//     reflector j only touches columns >= j and forming Q costs as many flops as the
//     factorization, not twice as many.
#include "tsqr_internal.h"

namespace tsqr {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Transpose-reduce over a full warp (C a power of two <= 32); see treduce16 in the
// factor kernel. The lane ends with the warp total of value idx.
template <int C>
__device__ __forceinline__ double treduce32(double (&v)[C], int lane, int &idx) {
  idx = 0;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int m = 16 >> s;
    const int cs = (C >> s) > 1 ? (C >> s) : 1;
    if (cs > 1) {
      const int half = cs >> 1;
      const bool up = (lane & m) != 0;
#pragma unroll
      for (int i = 0; i < C / 2; ++i) {
        if (i < half) {
          const double send = up ? v[i] : v[i + half];
          const double keep = up ? v[i + half] : v[i];
          v[i] = keep + __shfl_xor_sync(kFull, send, m);
        }
      }
      if (up) idx += half;
    } else {
      v[0] += __shfl_xor_sync(kFull, v[0], m);
    }
  }
  return v[0];
}

// Lowest lane that holds the total of value c after treduce32<C>.
template <int C>
__device__ __forceinline__ int treduce32_lane(int c) {
  int lane = 0;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int half = (C >> s) >> 1;
    if (half >= 1 && (c & half)) lane |= (16 >> s);
  }
  return lane;
}

template <int C>
__device__ __forceinline__ double treduce16(double (&v)[C], int hl, int &idx) {
  idx = 0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int m = 8 >> s;
    const int cs = (C >> s) > 1 ? (C >> s) : 1;
    if (cs > 1) {
      const int half = cs >> 1;
      const bool up = (hl & m) != 0;
#pragma unroll
      for (int i = 0; i < C / 2; ++i) {
        if (i < half) {
          const double send = up ? v[i] : v[i + half];
          const double keep = up ? v[i + half] : v[i];
          v[i] = keep + __shfl_xor_sync(kFull, send, m);
        }
      }
      if (up) idx += half;
    } else {
      v[0] += __shfl_xor_sync(kFull, v[0], m);
    }
  }
  return v[0];
}

constexpr int kWarpRows = 16;  // rows per lane in k_apply_warp: tiles of at most 512 rows

// ------------------------------------------------------------- one warp per job
template <int KM>
__global__ void __launch_bounds__(128) k_apply_warp(const ApplyParams p, int njobs) {
  extern __shared__ __align__(16) double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int jid = blockIdx.x * 4 + warp;
  if (jid >= njobs) return;  // warp-uniform; this kernel uses no block barrier
  const int n = p.n, k = p.k, ldt = p.ldt;
  double *Bt = sm + (size_t)warp * ((size_t)ldt + n) * KM;  // tile rows, column-major
  double *PR = Bt + (size_t)ldt * KM;                        // pivot rows, PR[c*n + j]
  const JobDesc job = p.jobs[p.job0 + jid];
  const int64_t pr = job.piv_row;
  auto bcol = [&](int c) -> double * { return p.B + (int64_t)(p.col0 + c) * p.ldb; };

  for (int c = 0; c < k; ++c)
    for (int j = lane; j < n; j += 32) PR[c * n + j] = bcol(c)[pr + j];
  __syncwarp();

  const int nt = job.tile_count;
  for (int q = 0; q < nt; ++q) {
    const int tt = p.trans ? q : nt - 1 - q;
    const TileDesc td = p.tiles[job.tile_begin + tt];
    const int ht = td.nrows, kind = td.kind;
    const bool ge = (kind == GEQRT);
    const int64_t r0 = td.row0;
    for (int c = 0; c < k; ++c) {
      const double *src = bcol(c) + r0;
      for (int i = lane; i < ht; i += 32)
        Bt[c * ldt + i] = (ge && i < n) ? PR[c * n + i] : (p.formq ? 0.0 : src[i]);
    }
    __syncwarp();

    const double *Vt = p.V + r0;
    double xv[kWarpRows], xn[kWarpRows];
    {
      const int j0 = p.trans ? 0 : n - 1;
      int lo, hi;
      refl_rows(kind, j0, ht, lo, hi);
#pragma unroll
      for (int r = 0; r < kWarpRows; ++r) {
        const int i = lane + 32 * r;
        xv[r] = (i >= lo && i < hi) ? __ldg(Vt + i + (int64_t)j0 * p.ldv) : 0.0;
      }
    }
    for (int s = 0; s < n; ++s) {
      const int j = p.trans ? s : n - 1 - s;
      int lo, hi;
      refl_rows(kind, j, ht, lo, hi);
      if (s + 1 < n) {
        const int jn = p.trans ? s + 1 : n - 2 - s;
        int lo2, hi2;
        refl_rows(kind, jn, ht, lo2, hi2);
#pragma unroll
        for (int r = 0; r < kWarpRows; ++r) {
          const int i = lane + 32 * r;
          xn[r] = (i >= lo2 && i < hi2) ? __ldg(Vt + i + (int64_t)jn * p.ldv) : 0.0;
        }
      }
      const double tau = __ldg(p.tau + td.refl + j);
      const double sc = __ldg(p.scl + td.refl + j);
      double part[KM];
#pragma unroll
      for (int c = 0; c < KM; ++c) part[c] = 0.0;
#pragma unroll
      for (int r = 0; r < kWarpRows; ++r) {
        const int i = lane + 32 * r;
        if (i >= lo && i < hi) {
#pragma unroll
          for (int c = 0; c < KM; ++c)
            if (c < k) part[c] = fma(xv[r], Bt[c * ldt + i], part[c]);
        }
      }
      int idx;
      const double tot = treduce32<KM>(part, lane, idx);
      double cfv = 0.0;
      if ((lane & (32 / KM - 1)) == 0 && idx < k) {
        double *pp = ge ? &Bt[idx * ldt + j] : &PR[idx * n + j];
        const double piv = *pp;
        const double w = fma(sc, tot, piv);
        *pp = fma(-tau, w, piv);
        cfv = tau * sc * w;
      }
      double cf[KM];
#pragma unroll
      for (int c = 0; c < KM; ++c) cf[c] = __shfl_sync(kFull, cfv, treduce32_lane<KM>(c));
      __syncwarp();
#pragma unroll
      for (int r = 0; r < kWarpRows; ++r) {
        const int i = lane + 32 * r;
        if (i >= lo && i < hi) {
#pragma unroll
          for (int c = 0; c < KM; ++c)
            if (c < k) Bt[c * ldt + i] = fma(-cf[c], xv[r], Bt[c * ldt + i]);
        }
      }
      __syncwarp();
#pragma unroll
      for (int r = 0; r < kWarpRows; ++r) xv[r] = xn[r];
    }
    for (int c = 0; c < k; ++c) {
      double *dst = bcol(c) + r0;
      for (int i = lane; i < ht; i += 32) {
        if (ge && i < n)
          PR[c * n + i] = Bt[c * ldt + i];
        else
          dst[i] = Bt[c * ldt + i];
      }
    }
    __syncwarp();
  }
  for (int c = 0; c < k; ++c)
    for (int j = lane; j < n; j += 32) bcol(c)[pr + j] = PR[c * n + j];
}

// ------------------------------------------------------------ one CTA per job
constexpr int kWideThreads = 256;
constexpr int kWideCM = 2;                 // column slots per half-warp
constexpr int kWideCols = 16 * kWideCM;    // columns per pass

__global__ void __launch_bounds__(kWideThreads) k_apply_wide(const ApplyParams p) {
  extern __shared__ __align__(16) double sm[];
  const int n = p.n, ldt = p.ldt;
  const int pass_col = blockIdx.y * kWideCols;
  const int col0 = p.col0 + pass_col;
  const int kc = min(kWideCols, p.k - pass_col);
  double *Bt = sm;                               // ldt x kWideCols
  double *PR = Bt + (size_t)ldt * kWideCols;     // n x kWideCols
  double *Vc = PR + (size_t)n * kWideCols;       // 2 x ldt
  double *Pg = Vc + 2 * (size_t)ldt;             // kWideCols
  double *CF = Pg + kWideCols;                   // kWideCols
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int hw = tid >> 4, hl = tid & 15;
  const JobDesc job = p.jobs[p.job0 + blockIdx.x];
  const int64_t pr = job.piv_row;
  auto bcol = [&](int c) -> double * { return p.B + (int64_t)(col0 + c) * p.ldb; };

  for (int c = warp; c < kc; c += kWideThreads / 32)
    for (int j = lane; j < n; j += 32) PR[c * n + j] = bcol(c)[pr + j];
  __syncthreads();

  const int nt = job.tile_count;
  for (int q = 0; q < nt; ++q) {
    const int tt = p.trans ? q : nt - 1 - q;
    const TileDesc td = p.tiles[job.tile_begin + tt];
    const int ht = td.nrows, kind = td.kind;
    const bool ge = (kind == GEQRT);
    const int64_t r0 = td.row0;
    const double *Vt = p.V + r0;
    for (int c = warp; c < kc; c += kWideThreads / 32) {
      const double *src = bcol(c) + r0;
      for (int i = lane; i < ht; i += 32)
        Bt[(size_t)c * ldt + i] = (ge && i < n) ? PR[c * n + i] : (p.formq ? 0.0 : src[i]);
    }
    {
      const int j0 = p.trans ? 0 : n - 1;
      int lo, hi;
      refl_rows(kind, j0, ht, lo, hi);
      for (int i = lo + tid; i < hi; i += kWideThreads) Vc[i] = __ldg(Vt + i + (int64_t)j0 * p.ldv);
    }
    __syncthreads();

    for (int s = 0; s < n; ++s) {
      const int j = p.trans ? s : n - 1 - s;
      const int buf = s & 1;
      const double *vc = Vc + (size_t)buf * ldt;
      int lo, hi;
      refl_rows(kind, j, ht, lo, hi);
      // prefetch the next reflector's tail into registers (at most 2 rows per thread)
      double pf0 = 0.0, pf1 = 0.0;
      int lo2 = 0, hi2 = 0;
      if (s + 1 < n) {
        const int jn = p.trans ? s + 1 : n - 2 - s;
        refl_rows(kind, jn, ht, lo2, hi2);
        const int i0 = lo2 + tid, i1 = lo2 + tid + kWideThreads;
        if (i0 < hi2) pf0 = __ldg(Vt + i0 + (int64_t)jn * p.ldv);
        if (i1 < hi2) pf1 = __ldg(Vt + i1 + (int64_t)jn * p.ldv);
      }
      const int cs = p.formq ? max(0, j - col0) : 0;  // first column this reflector touches
      if (cs < kc) {
        // dot products of the reflector tail with the tile columns
        const int cb = cs + hw;
        if (cs + 2 * warp < kc) {
          double acc[kWideCM];
#pragma unroll
          for (int t = 0; t < kWideCM; ++t) acc[t] = 0.0;
          for (int i = lo + hl; i < hi; i += 16) {
            const double x = vc[i];
#pragma unroll
            for (int t = 0; t < kWideCM; ++t) {
              const int c = cb + 16 * t;
              if (c < kc) acc[t] = fma(x, Bt[(size_t)c * ldt + i], acc[t]);
            }
          }
          int idx;
          const double sres = treduce16<kWideCM>(acc, hl, idx);
          const int c = cb + 16 * idx;
          if ((hl & (16 / kWideCM - 1)) == 0 && c < kc) Pg[c] = sres;
        }
        __syncthreads();
        if (tid >= cs && tid < kc) {
          const double tau = __ldg(p.tau + td.refl + j);
          const double sc = __ldg(p.scl + td.refl + j);
          const int c = tid;
          double *pp = ge ? &Bt[(size_t)c * ldt + j] : &PR[c * n + j];
          const double piv = *pp;
          const double w = fma(sc, Pg[c], piv);
          *pp = fma(-tau, w, piv);
          CF[c] = tau * sc * w;
        }
        __syncthreads();
        if (cs + 1 + 2 * warp - 1 < kc) {
          double cf[kWideCM];
#pragma unroll
          for (int t = 0; t < kWideCM; ++t) {
            const int c = cb + 16 * t;
            cf[t] = (c < kc) ? CF[c] : 0.0;
          }
          for (int i = lo + hl; i < hi; i += 16) {
            const double x = vc[i];
#pragma unroll
            for (int t = 0; t < kWideCM; ++t) {
              const int c = cb + 16 * t;
              if (c < kc) {
                double *b = Bt + (size_t)c * ldt + i;
                *b = fma(-cf[t], x, *b);
              }
            }
          }
        }
      }
      if (s + 1 < n) {
        double *vn = Vc + (size_t)(buf ^ 1) * ldt;
        const int i0 = lo2 + tid, i1 = lo2 + tid + kWideThreads;
        if (i0 < hi2) vn[i0] = pf0;
        if (i1 < hi2) vn[i1] = pf1;
      }
      __syncthreads();
    }
    for (int c = warp; c < kc; c += kWideThreads / 32) {
      double *dst = bcol(c) + r0;
      for (int i = lane; i < ht; i += 32) {
        if (ge && i < n)
          PR[c * n + i] = Bt[(size_t)c * ldt + i];
        else
          dst[i] = Bt[(size_t)c * ldt + i];
      }
    }
    __syncthreads();
  }
  for (int c = warp; c < kc; c += kWideThreads / 32)
    for (int j = lane; j < n; j += 32) bcol(c)[pr + j] = PR[c * n + j];
}

template <int KM>
cudaError_t launch_warp_t(const ApplyParams &p, int njobs, cudaStream_t s) {
  const size_t bytes = sizeof(double) * 4 * ((size_t)p.ldt + p.n) * KM;
  cudaError_t e = cudaFuncSetAttribute(k_apply_warp<KM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return e;
  k_apply_warp<KM><<<(njobs + 3) / 4, 128, bytes, s>>>(p, njobs);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_apply(const ApplyParams &p, int njobs, cudaStream_t s) {
  if (njobs <= 0 || p.k <= 0) return cudaSuccess;
  if (p.k <= 8 && p.ldt <= 32 * kWarpRows) {
    if (p.k == 1) return launch_warp_t<1>(p, njobs, s);
    if (p.k == 2) return launch_warp_t<2>(p, njobs, s);
    if (p.k <= 4) return launch_warp_t<4>(p, njobs, s);
    return launch_warp_t<8>(p, njobs, s);
  }
  if (p.ldt > 2 * kWideThreads) return cudaErrorInvalidValue;
  const size_t bytes = sizeof(double) * ((size_t)p.ldt * kWideCols + (size_t)p.n * kWideCols +
                                         2 * (size_t)p.ldt + 2 * kWideCols);
  cudaError_t e = cudaFuncSetAttribute(k_apply_wide, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return e;
  dim3 grid(njobs, (p.k + kWideCols - 1) / kWideCols);
  k_apply_wide<<<grid, kWideThreads, bytes, s>>>(p);
  return cudaGetLastError();
}

}  // namespace tsqr
