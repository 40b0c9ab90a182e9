// TSQR factorization kernels (sm_103a), FP64 and FP32 instantiations. The job code they
// share with the resident kernel is in factor_job.cuh; the notes below describe it.
//
// One CTA runs one job (a chain of tiles sharing n pivot rows, see tsqr_internal.h).
// Each tile is staged in shared memory and factored column by column with Householder
// reflections (paper §2.2); the pivot row of reflector j is the tile's own row j (GEQRT,
// a leaf) or row j of the job's running triangle R held in global memory (TSQRT: the
// flat-tree step [R; tile], TTQRT: the tree combine [R; R_child], paper §2.3).
//
// GB300 design notes. FP64 runs on a narrow pipe (2 DFMA/clk/SM: each of the four SM
// sub-partitions takes one FP64 warp instruction per 64 cycles) and a warp instruction
// costs the same with masked lanes, so the kernel keeps warps full, spends FP64 issue
// slots only on the factorization itself, and spreads them evenly over sub-partitions:
//   * per column step j the dot products p_k = sum_i b_ij b_ik (k > j) are one Gram-row
//     pass, so one reduction per step;
//   * a worker half-warp owns columns; each lane walks 1/16 of the rows, so a value is
//     reduced over only 16 lanes, by a transpose-reduce that spends about one DADD per
//     value instead of four;
//   * reflectors are stored unscaled with (tau, scale) beside them, so the update of a
//     trailing element is exactly one DFMA: b_ik -= (tau*scale*w_k) * b_ij;
//   * every warp issues exactly as many column slots as it owns at each step: a
//     predicated-off DFMA still occupies the FP64 pipe, so the column guards are
//     warp-uniform branches, not predicates;
//   * the reflector's scalar chain runs on its own warp, overlapped with the dot
//     products (run_job below), and the column dealing rotates with the step so that no
//     sub-partition's FP64 pipe carries more than its share.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "cluster_sync.cuh"
#include "factor_job.cuh"
#include "tsqr_internal.h"
#include "warp_reduce.cuh"

namespace tsqr {
namespace {

// ------------------------------------ FP32 chains: compact-WY panels on tensor cores
// The same chain job as run_job_f32s (same register tile, same reflector storage and R),
// blocked: the columns are factored in panels of 16 (one register slot), each column step
// touching only the panel's columns, and the panel's 16 reflectors are then applied to the
// trailing columns at once in compact-WY form (paper §2.2: the blocked Householder update):
//   Q_panel = H_c0 ... H_c0+15 = I - V T V^T,   C <- Q_panel^T C = C - V (T^T (V^T C)),
// T upper triangular from the forward recurrence T[0:j, j] = -tau_j T[0:j, 0:j] (V^T v_j)[0:j].
// V^T C and V (T^T W) are dense contractions and run on the tensor cores as 3xTF32
// (mma.sync m16n8k8, every FP32 operand split as hi + lo with hi = tf32(x),
// lo = tf32(x - hi); products hi*hi + hi*lo + lo*hi accumulated in FP32, which keeps FP32
// accuracy; Ootomo & Yokota 2022). The trailing columns pass through shared memory in
// chunks of 32 (two register slots) for the products.
// For a leaf tile (GEQRT) v_j is 1 at tile row j and zero above; for a triangle-on-tile
// step (TSQRT) v_j is 1 at pivot row j of the chain's R (shared memory) and scale_j times
// the tile's column j below, so V^T C gains R's pivot rows and R's rows take -T^T W.
constexpr int kWyPanel = 16;
constexpr int kWyChunk = 32;
constexpr int kWyLd = kF32TileRows + 4;  // column stride of V and of a chunk (bank spread)
constexpr int kWyLdT = kWyPanel + 4;     // row stride of V^T and column stride of W'

__device__ __forceinline__ uint32_t tf32_of(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo) {
  hi = tf32_of(x);
  lo = tf32_of(x - __uint_as_float(hi));
}
// d += a b for one m16n8k8 TF32 tile (a: 16x8 row-major fragment, b: 8x8 column-major)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// 3xTF32: d += a b from FP32 fragments (the small cross terms first)
__device__ __forceinline__ void mma_3xtf32(float (&d)[4], const float (&a)[4], const float (&b)[2]) {
  uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
  for (int q = 0; q < 4; ++q) tf32_split(a[q], ah[q], al[q]);
#pragma unroll
  for (int q = 0; q < 2; ++q) tf32_split(b[q], bh[q], bl[q]);
  mma_tf32(d, al, bh);
  mma_tf32(d, ah, bl);
  mma_tf32(d, ah, bh);
}

template <int CPT>
__device__ __forceinline__ void run_job_f32wy(const FactorParamsT<float> &p, const JobDesc job, unsigned char *smraw) {
  float *sm = reinterpret_cast<float *>(smraw);
  const int n = p.n, nc = p.nc;
  const int ncp = (nc + 7) & ~7;
  float *xcol = sm;
  float *PC = xcol + kF32TileRows;
  float *PVb = PC + ncp;
  const int ldr = ncp + 1;
  float *Rs = PVb + 2 * ncp;              // R(i, c) at Rs[i * ldr + c]
  float *VS = Rs + (size_t)n * ldr;       // V, column q at VS[q * kWyLd + i]
  float *VT = VS + kWyPanel * kWyLd;      // V again, row-major: VT[i * kWyLdT + q]
  float *CT = VT + kF32TileRows * kWyLdT; // a chunk of trailing columns, CT[c * kWyLd + i]
  float *WP = CT + kWyChunk * kWyLd;      // two partial V^T C (K halves), WP[h][c * 16 + q]
  float *WT = WP + 2 * kWyPanel * kWyChunk;  // W' = T^T W, WT[c * kWyLdT + q]
  float *GG = WT + kWyChunk * kWyLdT;     // G = V^T V, GG[a * 17 + b]
  float *TT = GG + kWyPanel * (kWyPanel + 1);  // T, TT[i * 17 + j]
  float *TAU = TT + kWyPanel * (kWyPanel + 1);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int hw = tid >> 4, hl = tid & 15;
  const int g = lane >> 2, tg = lane & 3;  // mma fragment coordinates
  const int64_t pr = job.piv_row;
  float v[CPT][kF32Rpt];

  for (int tt = 0; tt < job.tile_count; ++tt) {
    const TileDesc td = p.tiles[job.tile_begin + tt];
    const int ht = td.nrows;
    const int64_t r0 = td.row0;
    const bool ge = (td.kind == GEQRT);
#pragma unroll
    for (int t = 0; t < CPT; ++t) {
      const int c = hw + 16 * t;
#pragma unroll
      for (int r = 0; r < kF32Rpt; ++r) {
        const int i = hl + 16 * r;
        float val = 0.f;
        if (c < nc && i < ht)
          val = (c < n) ? (float)__ldg(p.A + r0 + i + (int64_t)c * p.lda)
                        : __ldcg(p.B + r0 + i + (int64_t)(c - n) * p.ldb);
        v[t][r] = val;
      }
    }
    __syncthreads();

#pragma unroll
    for (int pp = 0; pp < CPT; ++pp) {  // panel pp = columns 16 pp .. 16 pp + 15 (register slot pp)
      const int c0 = kWyPanel * pp;
      if (c0 >= n) break;
      const int pend = min(n, c0 + kWyPanel);
      // ---- the panel's column steps (only the panel's columns are touched)
      for (int j = c0; j < pend; ++j) {
        const int jl = j & 15;
        float *PV = ge ? PVb + (j & 1) * ncp : Rs + j * ldr;
        if (hw == jl)
#pragma unroll
          for (int r = 0; r < kF32Rpt; ++r) xcol[hl + 16 * r] = v[pp][r];
        if (ge && hl == jl) {  // pivot row j (= tile row j) of the panel's columns
          const int c = hw + c0;
#pragma unroll
          for (int r = 0; r < kF32Rpt; ++r)
            if (r == pp && c >= j && c < pend) PV[c] = v[pp][r];
        }
        __syncthreads();
        float x[kF32Rpt];
#pragma unroll
        for (int r = 0; r < kF32Rpt; ++r) {
          const int i = hl + 16 * r;
          x[r] = (ge && i <= j) ? 0.f : xcol[i];
        }
        {  // Gram row over the panel (column c = c0 + hw; c == j gives the tail's squared norm)
          float acc = 0.f;
#pragma unroll
          for (int r = 0; r < kF32Rpt; ++r) acc = fmaf(x[r], v[pp][r], acc);
#pragma unroll
          for (int o = 8; o >= 1; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
          const int c = c0 + hw;
          if (hl == 0 && c >= j && c < pend) PC[c] = acc;
        }
        __syncthreads();
        if (warp == 0) {
          const Refl<float> rf = reflector<float>(PV[j], PC[j]);
          __syncwarp();  // every lane has read PC[j] before lane 0 replaces it
          const int c = j + 1 + lane;
          if (c < pend) {
            const float pk = PV[c];
            const float w = fmaf(rf.scale, PC[c], pk);
            PC[c] = rf.ts * w;
            PV[c] = fmaf(-rf.tau, w, pk);
          }
          if (lane == 0) {
            PV[j] = rf.beta;
            p.tau[td.refl + j] = rf.tau;
            p.scl[td.refl + j] = rf.scale;
            TAU[j - c0] = rf.tau;
            PC[j] = rf.scale;  // kept for V's scaling below
          }
        }
        __syncthreads();
        {
          const int c = c0 + hw;
          if (c > j && c < pend) {
            const float cf = PC[c];
#pragma unroll
            for (int r = 0; r < kF32Rpt; ++r) v[pp][r] = fmaf(-cf, x[r], v[pp][r]);
          }
          if (ge && hl == jl && c >= j && c < pend)
#pragma unroll
            for (int r = 0; r < kF32Rpt; ++r)
              if (r == (j >> 4)) v[pp][r] = PV[c];
        }
      }
      if (pend >= nc) continue;  // no trailing columns
      __syncthreads();
      // ---- V (scaled reflectors) in both layouts, then G = V^T V and T
      {
        const int q = hw, c = c0 + hw;
        const float sc = (c < pend) ? PC[c] : 0.f;
#pragma unroll
        for (int r = 0; r < kF32Rpt; ++r) {
          const int i = hl + 16 * r;
          float val;
          if (c >= pend)
            val = 0.f;
          else if (ge)
            val = (i < c) ? 0.f : (i == c ? 1.f : sc * v[pp][r]);
          else
            val = sc * v[pp][r];
          VS[q * kWyLd + i] = val;
          VT[i * kWyLdT + q] = val;
        }
      }
      __syncthreads();
      {  // G[a][b] = v_a . v_b (the TSQRT unit pivots add the identity)
        const int a = tid >> 4, b = tid & 15;
        float acc = (!ge && a == b) ? 1.f : 0.f;
        for (int i = 0; i < kF32TileRows; ++i) acc = fmaf(VS[a * kWyLd + i], VS[b * kWyLd + i], acc);
        GG[a * 17 + b] = acc;
      }
      __syncthreads();
      if (tid < kWyPanel) {  // T column by column; thread i owns row i and reads only it
        const int i = tid, nb = pend - c0;
        for (int j = 0; j < kWyPanel; ++j) {
          float tv = 0.f;
          if (j < nb) {
            if (i == j) {
              tv = TAU[j];
            } else if (i < j) {
              float s2 = 0.f;
              for (int l = i; l < j; ++l) s2 = fmaf(TT[i * 17 + l], GG[l * 17 + j], s2);
              tv = -TAU[j] * s2;
            }
          }
          TT[i * 17 + j] = tv;
        }
      }
      __syncthreads();
      // ---- the trailing columns, two register slots (32 columns) at a time
#pragma unroll
      for (int ts = 0; ts < CPT; ts += 2) {
        if (ts + 1 <= pp) continue;          // chunk entirely inside the factored columns
        const int cb = 16 * ts;              // first column of the chunk
        // stage: slots ts and ts + 1 (columns not past the panel are zeroed: V^T C of them
        // is not needed and they must stay unchanged)
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int t = ts + u;
          if (t >= CPT) continue;
          const int c = hw + 16 * t;
#pragma unroll
          for (int r = 0; r < kF32Rpt; ++r)
            CT[(16 * u + hw) * kWyLd + hl + 16 * r] = (c >= pend && c < nc) ? v[t][r] : 0.f;
        }
        __syncthreads();
        {  // V^T C: warp w takes columns 8 (w & 3) .. + 7 and rows 64 (w >> 2) .. + 63
          const int nb = 8 * (warp & 3), kh = warp >> 2;
          float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
          for (int kk = 0; kk < 8; ++kk) {
            const int kb = 64 * kh + 8 * kk;
            const float a[4] = {VS[g * kWyLd + kb + tg], VS[(g + 8) * kWyLd + kb + tg], VS[g * kWyLd + kb + tg + 4],
                                VS[(g + 8) * kWyLd + kb + tg + 4]};
            const float b[2] = {CT[(nb + g) * kWyLd + kb + tg], CT[(nb + g) * kWyLd + kb + tg + 4]};
            mma_3xtf32(d, a, b);
          }
          float *w = WP + kh * kWyPanel * kWyChunk;
          w[(nb + 2 * tg) * kWyPanel + g] = d[0];
          w[(nb + 2 * tg + 1) * kWyPanel + g] = d[1];
          w[(nb + 2 * tg) * kWyPanel + g + 8] = d[2];
          w[(nb + 2 * tg + 1) * kWyPanel + g + 8] = d[3];
        }
        __syncthreads();
        // W = the two halves (+ R's pivot rows for a TSQRT tile); W' = T^T W; R's pivot
        // rows take -W' (the unit pivots of V)
        for (int e = tid; e < kWyPanel * kWyChunk; e += kThreads) {
          const int q = e & 15, c = e >> 4;
          const int col = cb + c;
          float wsum = 0.f;
          for (int l = 0; l <= q; ++l) {
            float wl = WP[c * kWyPanel + l] + WP[kWyPanel * kWyChunk + c * kWyPanel + l];
            if (!ge && col >= pend && col < nc && c0 + l < pend) wl += Rs[(c0 + l) * ldr + col];
            wsum = fmaf(TT[l * 17 + q], wl, wsum);
          }
          WT[c * kWyLdT + q] = wsum;
        }
        __syncthreads();
        if (!ge)
          for (int e = tid; e < kWyPanel * kWyChunk; e += kThreads) {
            const int q = e & 15, c = e >> 4, col = cb + c;
            if (col >= pend && col < nc && c0 + q < pend) Rs[(c0 + q) * ldr + col] -= WT[c * kWyLdT + q];
          }
        {  // C -= V W': warp w takes rows 16 w .. 16 w + 15, all 32 columns
          const int mb = 16 * warp;
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            const int nb = 8 * nt;
            float d[4] = {CT[(nb + 2 * tg) * kWyLd + mb + g], CT[(nb + 2 * tg + 1) * kWyLd + mb + g],
                          CT[(nb + 2 * tg) * kWyLd + mb + g + 8], CT[(nb + 2 * tg + 1) * kWyLd + mb + g + 8]};
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              const int kb = 8 * kk;
              const float a[4] = {-VT[(mb + g) * kWyLdT + kb + tg], -VT[(mb + g + 8) * kWyLdT + kb + tg],
                                  -VT[(mb + g) * kWyLdT + kb + tg + 4], -VT[(mb + g + 8) * kWyLdT + kb + tg + 4]};
              const float b[2] = {WT[(nb + g) * kWyLdT + kb + tg], WT[(nb + g) * kWyLdT + kb + tg + 4]};
              mma_3xtf32(d, a, b);
            }
            CT[(nb + 2 * tg) * kWyLd + mb + g] = d[0];
            CT[(nb + 2 * tg + 1) * kWyLd + mb + g] = d[1];
            CT[(nb + 2 * tg) * kWyLd + mb + g + 8] = d[2];
            CT[(nb + 2 * tg + 1) * kWyLd + mb + g + 8] = d[3];
          }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int t = ts + u;
          if (t >= CPT) continue;
          const int c = hw + 16 * t;
          if (c >= pend && c < nc)
#pragma unroll
            for (int r = 0; r < kF32Rpt; ++r) v[t][r] = CT[(16 * u + hw) * kWyLd + hl + 16 * r];
        }
        __syncthreads();
      }
    }
    __syncthreads();
    if (ge) {
#pragma unroll
      for (int t = 0; t < CPT; ++t) {
        const int c = hw + 16 * t;
#pragma unroll
        for (int r = 0; r < kF32Rpt; ++r) {
          const int i = hl + 16 * r;
          if (c < nc && i < n && (i <= c || c >= n)) Rs[i * ldr + c] = v[t][r];
        }
      }
    }
#pragma unroll
    for (int t = 0; t < CPT; ++t) {
      const int c = hw + 16 * t;
      if (c >= nc) continue;
      float *dst = (c < n) ? p.V + r0 + (int64_t)c * p.ldv : p.B + r0 + (int64_t)(c - n) * p.ldb;
#pragma unroll
      for (int r = 0; r < kF32Rpt; ++r) {
        const int i = hl + 16 * r;
        if (i < ht) dst[i] = v[t][r];
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < n * nc; e += kThreads) {
    const int i = e % n, c = e / n;
    if (i <= c || c >= n) {
      float *dst = (c < n) ? p.V + pr + i + (int64_t)c * p.ldv : p.B + pr + i + (int64_t)(c - n) * p.ldb;
      *dst = Rs[i * ldr + c];
    }
  }
  __syncthreads();
}

// ------------------------------------------------- cluster tier: pipelined tree levels
// Three binary levels of the reduction tree in one launch of thread-block clusters of
// kClusterSize CTAs (the GPU analogue of the paper's hierarchical tree, §2.3 and §3:
// combines inside a cluster exchange their triangles on chip, through distributed shared
// memory, and only the cluster's root goes on to the next level across the grid).
//
// A combine [R1; R2] -> R (TTQRT) reads at its column step j only row j of each child's
// triangle (reflector j pivots on row j of R1 and has its tail in rows 0..j of R2, which
// steps < j never touched), and that row is final once the child has finished its own step
// j. So a parent starts step j as soon as both children have published j + 1 finished
// steps: the levels of a cluster run as a pipeline, and three levels cost about n + 3 column
// steps instead of 3n. Each CTA keeps its pivot triangle row-major in shared memory (the
// rows of its output triangle as they become final); a parent copies a child's row j from
// the child's shared memory (mapa + ld.shared::cluster) after an acquire load of the child's
// progress counter, which the child advances with a release store at cluster scope. Every
// wait is bounded: past the limit the CTA sets the device error word's timeout bit and
// stops waiting, so the launch always ends.

// One combine job of the cluster tier (a binary node: one TTQRT tile of n rows), run by
// the factor kernel's eight warps plus a ninth, the copy warp.
// Shared memory: T, the tile child's triangle (column-major, ld n, nc columns); PC, the
// step's dot products then coefficients; P, the pivot triangle, row-major (ld ncp), whose
// row j becomes this node's output row j at step j. `done` counts this CTA's finished
// steps; `gave_up` (shared) is set once a wait timed out.
// Column step j reads only rows 0..j of T and row j of P, so while the other warps run
// step j the copy warp waits for the in-cluster children to finish their step j + 1 and
// copies their row j + 1 in: the distributed-shared-memory latency overlaps the step, and
// a step keeps the factor kernel's barriers (two named, one full).
constexpr int kCopyWarp = kScalarWarp + 1;
constexpr int kClusterThreads = kThreads + 32;

template <int CMAX>
__device__ __forceinline__ void run_node_cluster(const FactorParamsT<double> &p, const JobDesc job, const int c0,
                                                 const int c1, unsigned char *smraw, unsigned *done, int *gave_up,
                                                 int32_t *err) {
  using R = double;
  R *sm = reinterpret_cast<R *>(smraw);
  const int n = p.n, nc = p.nc, ldt = n;
  const int ncp = (nc + 7) & ~7;
  R *T = sm;
  R *PC = T + (size_t)nc * ldt;
  R *P = PC + ncp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool sw = (warp == kScalarWarp), cw = (warp == kCopyWarp);
  const int hl = tid & 15, hsub = (tid >> 4) & 1;
  const TileDesc td = p.tiles[job.tile_begin];
  const int64_t pr = job.piv_row, r0 = td.row0;
  auto gptr = [&](int64_t row, int c) -> R * {
    return (c < n) ? p.V + row + (int64_t)c * p.ldv : p.B + row + (int64_t)(c - n) * p.ldb;
  };
  constexpr int PCN = (job_nc_max(CMAX) + 31) / 32;
  TSQR_CHECK_OR_SKIP(job.tile_count == 1 && td.kind == TTQRT && td.nrows == n && td.off == 0 && pr >= 0 && r0 >= 0 &&
                         (p.rows == 0 || (pr + n <= p.rows && r0 + n <= p.rows)) && td.refl >= 0 &&
                         (p.nrefl == 0 || td.refl + n <= p.nrefl) && c0 >= -1 && c0 < kClusterSize && c1 >= -1 &&
                         c1 < kClusterSize && nc <= job_nc_max(CMAX),
                     p.err)
  const uint32_t a_done = smem_u32(done), a_P = smem_u32(P);
  // the copy warp: wait until the in-cluster children have finished `steps` steps (every
  // lane polls, so each lane's later loads are ordered after its own acquire), then copy
  // their row `row` into P / T
  auto fetch_row = [&](int row) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int ch = q == 0 ? c0 : c1;
      if (ch < 0) continue;  // warp-uniform
      if (!*gave_up) {
        const uint32_t a = cluster_map(a_done, ch);
        uint32_t it = 0;
        while (ld_acquire_cluster_u32(a) < (uint32_t)(row + 1)) {
          if (++it > kClusterSpinLimit) {
            if (lane == 0) atomicOr(err, kErrTimeout);
            *gave_up = 1;
            break;
          }
          __nanosleep(32);
        }
      }
      __syncwarp();
      for (int c = row + lane; c < nc; c += 32) {
        const R v = ld_cluster_f64(cluster_map(a_P + (uint32_t)(sizeof(R) * ((size_t)row * ncp + c)), ch));
        if (q == 0)
          P[(size_t)row * ncp + c] = v;
        else
          T[(size_t)c * ldt + row] = v;
      }
    }
  };

  // triangles complete in global memory (an earlier launch's) are staged whole; row 0 of
  // in-cluster children before the first step
  if (c1 < 0)
    for (int c = warp; c < nc; c += kClusterThreads / 32) {
      const int lim = (c < n) ? min(n, c + 1) : n;
      warp_copy(T + (size_t)c * ldt, gptr(r0, c), lim, lane, [](const double *q) { return __ldcg(q); },
                [](const double2 *q) { return __ldcg(q); });
    }
  if (c0 < 0)
    for (int e = tid; e < n * nc; e += kClusterThreads) {
      const int i = e % n, c = e / n;
      if (c >= i) P[(size_t)i * ncp + c] = __ldcg(gptr(pr + i, c));
    }
  if (cw) fetch_row(0);
  __syncthreads();

  for (int j = 0; j < n; ++j) {
    R *PV = P + (size_t)j * ncp;  // the pivot row of this step
    const int lo = 0, hi = j + 1;  // reflector j's tail: rows 0..j of the child's triangle
    if (cw) {
      if (j + 1 < n) fetch_row(j + 1);
    } else if (!sw) {
      const int rw = (warp + j) % kWorkerWarps;
      const int v = 2 * rw + hsub;
      gram_row_dispatch<CMAX, R>(T, ldt, j, j + 1, nc, lo, hi, v, hl, rw, PC);
      bar_arrive_n(1, kThreads);
      bar_sync_n(2, kThreads);
      update_dispatch<CMAX, R>(T, ldt, j, j + 1, nc, lo, hi, v, hl, rw, PC);
    } else {
      const R *Tj = T + (size_t)j * ldt;
      R a0 = R(0), a1 = R(0);
      int i = lo + lane;
      for (; i + 32 < hi; i += 64) {
        const R x0 = Tj[i], x1 = Tj[i + 32];
        a0 = fma(x0, x0, a0);
        a1 = fma(x1, x1, a1);
      }
      if (i < hi) a0 = fma(Tj[i], Tj[i], a0);
      R s2 = a0 + a1;
#pragma unroll
      for (int m = 16; m >= 1; m >>= 1) s2 += __shfl_xor_sync(kFull, s2, m);
      const Refl<R> rf = reflector<R>(PV[j], s2);
      bar_sync_n(1, kThreads);
      R pk[PCN];
#pragma unroll
      for (int q = 0; q < PCN; ++q) {
        const int c = j + 1 + lane + 32 * q;
        if (c < nc) {
          const R p0 = PV[c];
          const R w = fma(rf.scale, PC[c], p0);
          PC[c] = rf.ts * w;
          pk[q] = fma(-rf.tau, w, p0);
        }
      }
      bar_arrive_n(2, kThreads);
      // the output row j: kept in shared memory for the parent, and written to the pivot
      // rows in global memory (the next launch's input, the apply kernels' R)
#pragma unroll
      for (int q = 0; q < PCN; ++q) {
        const int c = j + 1 + lane + 32 * q;
        if (c < nc) {
          PV[c] = pk[q];
          *gptr(pr + j, c) = pk[q];
        }
      }
      if (lane == 0) {
        PV[j] = rf.beta;
        *gptr(pr + j, j) = rf.beta;
        p.tau[td.refl + j] = rf.tau;
        p.scl[td.refl + j] = rf.scale;
      }
      __syncwarp();
    }
    __syncthreads();
    if (tid == 0) st_release_cluster_u32(a_done, (uint32_t)(j + 1));
  }
  // the child's triangle becomes this node's triangular reflector block
  for (int c = warp; c < nc; c += kClusterThreads / 32) {
    const int lim = (c < n) ? min(n, c + 1) : n;
    warp_copy(gptr(r0, c), T + (size_t)c * ldt, lim, lane, [](const double *q) { return *q; },
              [](const double2 *q) { return *q; });
  }
}

template <int CMAX>
__global__ void __launch_bounds__(kClusterThreads, 2) k_factor_cluster(const FactorParamsT<double> p,
                                                                       const ClusterSlot *__restrict__ slots,
                                                                       int32_t *err) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ unsigned s_done;
  __shared__ int s_gave_up;
  const ClusterSlot sl = slots[blockIdx.x];
  if (threadIdx.x == 0) {
    s_done = 0;
    s_gave_up = 0;
  }
  cluster_barrier();  // every counter is initialised before any CTA of the cluster polls it
  if (sl.job >= 0)
    run_node_cluster<CMAX>(p, p.jobs[sl.job], sl.child[0], sl.child[1], smraw, &s_done, &s_gave_up, err);
  cluster_barrier();  // no CTA leaves while a parent may still read its shared memory
}

// MINB = CTAs resident per SM the launch is planned for (2, or 3 with shorter tiles: more
// independent column-step sequences per SM hide more of each step's serial latency).
template <int CMAX, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_factor(const FactorParamsT<double> p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  run_job<CMAX, true>(p, p.jobs[p.job0 + blockIdx.x], smraw);
}

// ----------------------------------------------------------- batched persistent kernel

// WY: the build that can run mixed chains by compact-WY panels (run_job_f32wy); the
// kernel without it keeps its register budget for the other job kinds.
template <int CMAX, bool WY>
__global__ void __launch_bounds__(kThreads, 2) k_factor_batch(const BatchParams bp) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_job, s_go;
  for (;;) {
    if (threadIdx.x == 0) s_job = atomicAdd(bp.queue, 1);
    __syncthreads();
    int jb = s_job;
    __syncthreads();
    if (jb >= bp.nchains) return;
    for (;;) {
      const BatchJob bj = bp.jobs[jb];
      const BatchInst in = bp.inst[bj.inst];
      const JobDesc jd{bj.piv_row, bj.tile_begin, bj.tile_count};
      const bool chain = jb < bp.nchains;
      if (chain && in.mixed) {
        FactorParamsT<float> fp{};
        fp.A = in.A;
        fp.lda = in.lda;
        fp.V = static_cast<float *>(in.V);
        fp.ldv = in.ldv;
        fp.tiles = bp.tiles;
        fp.tau = static_cast<float *>(in.tau);
        fp.scl = static_cast<float *>(in.scl);
        fp.n = in.n;
        fp.nc = in.n;
        fp.ldt = in.ldt;
        if (WY && in.wy) {  // compact-WY panels, 3xTF32 tensor-core trailing updates
          switch (in.n <= 32 ? 2 : (in.n <= 64 ? 4 : 8)) {
            case 2: if constexpr (WY && CMAX >= 2) run_job_f32wy<2>(fp, jd, smraw); break;
            case 4: if constexpr (WY && CMAX >= 4) run_job_f32wy<4>(fp, jd, smraw); break;
            default: if constexpr (WY && CMAX >= 8) run_job_f32wy<8>(fp, jd, smraw); break;
          }
        } else {
          switch (in.n <= 16 ? 1 : (in.n <= 32 ? 2 : (in.n <= 64 ? 4 : 8))) {
            case 1: run_job_f32s<1>(fp, jd, smraw); break;
            case 2: if (CMAX >= 2) run_job_f32s<(CMAX >= 2 ? 2 : 1)>(fp, jd, smraw); break;
            case 4: if (CMAX >= 4) run_job_f32s<(CMAX >= 4 ? 4 : 1)>(fp, jd, smraw); break;
            default: if (CMAX >= 8) run_job_f32s<(CMAX >= 8 ? 8 : 1)>(fp, jd, smraw); break;
          }
        }
        // hand the chain's triangle to the FP64 tree storage
        const float *Vs = static_cast<const float *>(in.V) + bj.piv_row;
        for (int e = threadIdx.x; e < in.n * in.n; e += blockDim.x) {
          const int i = e % in.n, j = e / in.n;
          if (i <= j) in.V64[bj.row64 + i + (int64_t)j * in.ldv64] = (double)__ldcg(Vs + i + (int64_t)j * in.ldv);
        }
        __syncthreads();
      } else {
        FactorParamsT<double> fp{};
        fp.A = in.A;
        fp.lda = in.lda;
        fp.V = chain ? static_cast<double *>(in.V) : in.V64;
        fp.ldv = chain ? in.ldv : in.ldv64;
        fp.B = in.B;
        fp.ldb = in.ldb;
        fp.tiles = bp.tiles;
        fp.tau = chain ? static_cast<double *>(in.tau) : in.tau64;
        fp.scl = chain ? static_cast<double *>(in.scl) : in.scl64;
        fp.n = in.n;
        fp.nc = in.n + in.k;
        fp.ldt = chain ? in.ldt : in.ldt_tree;
        run_job<CMAX, true>(fp, jd, smraw);
      }
      if (bj.parent < 0) {
        __threadfence();
        finish_instance(in, bj.row64, smraw);
        break;
      }
      // publish this job's triangle, then arrive at the parent; the last child combines
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) s_go = (atomicAdd(bp.counters + bj.parent, 1) == bp.jobs[bj.parent].nchild - 1);
      __syncthreads();
      const int go = s_go;
      __syncthreads();
      if (!go) break;
      __threadfence();
      jb = bj.parent;
    }
  }
}

template <int CMAX, int MINB>
cudaError_t launch_factor_t(const FactorParamsT<double> &p, int njobs, cudaStream_t s) {
  const size_t bytes = factor_smem_bytes(p.nc, p.ldt, sizeof(double));
  cudaError_t e = cudaFuncSetAttribute(k_factor<CMAX, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return e;
  k_factor<CMAX, MINB><<<njobs, kThreads, bytes, s>>>(p);
  return cudaGetLastError();
}

template <int MINB>
cudaError_t launch_factor_c(const FactorParamsT<double> &p, int njobs, cudaStream_t s) {
  if (p.nc <= 16) return launch_factor_t<1, MINB>(p, njobs, s);
  if (p.nc <= 32) return launch_factor_t<2, MINB>(p, njobs, s);
  if (p.nc <= 64) return launch_factor_t<4, MINB>(p, njobs, s);
  return launch_factor_t<8, MINB>(p, njobs, s);
}

cudaError_t launch_factor_any(const FactorParamsT<double> &p, int njobs, int ctas_per_sm, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  // up to 16 columns (one column slot per half-warp) a step keeps at most half of a CTA's
  // worker warps busy: the 64-register build lets a fourth CTA join where its tile fits
  // (the plan, made for three, is unchanged)
  if (ctas_per_sm >= 3 && p.nc <= 16) return launch_factor_t<1, 4>(p, njobs, s);
  if (ctas_per_sm >= 3) return launch_factor_c<3>(p, njobs, s);
  return launch_factor_c<2>(p, njobs, s);
}

template <int CMAX>
cudaError_t launch_cluster_t(const FactorParamsT<double> &p, const ClusterSlot *slots, int nclusters, int32_t *err,
                             cudaStream_t s) {
  const int ncp = (p.nc + 7) & ~7;
  const size_t bytes = sizeof(double) * ((size_t)p.nc * p.n + ncp + (size_t)p.n * ncp);
  cudaError_t e = cudaFuncSetAttribute(k_factor_cluster<CMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nclusters * kClusterSize));
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kClusterSize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_factor_cluster<CMAX>, p, slots, err);
}

__device__ int32_t g_error_word;

}  // namespace

size_t f32wy_smem_extra_bytes() {
  return sizeof(float) * ((size_t)kWyPanel * kWyLd + (size_t)kF32TileRows * kWyLdT + (size_t)kWyChunk * kWyLd +
                          2 * (size_t)kWyPanel * kWyChunk + (size_t)kWyChunk * kWyLdT +
                          2 * (size_t)kWyPanel * (kWyPanel + 1) + kWyPanel);
}

size_t cluster_smem_bytes(int n, int nc, size_t optin_per_block) {
  const size_t ncp = (size_t)((nc + 7) & ~7);
  const size_t b = sizeof(double) * ((size_t)nc * n + ncp + (size_t)n * ncp);
  return b <= optin_per_block ? b : 0;
}

cudaError_t launch_factor_cluster(const FactorParamsT<double> &p, const ClusterSlot *slots, int nclusters,
                                  int32_t *err, cudaStream_t s) {
  if (nclusters <= 0) return cudaSuccess;
  if (p.nc <= 16) return launch_cluster_t<1>(p, slots, nclusters, err, s);
  if (p.nc <= 32) return launch_cluster_t<2>(p, slots, nclusters, err, s);
  if (p.nc <= 64) return launch_cluster_t<4>(p, slots, nclusters, err, s);
  return launch_cluster_t<8>(p, slots, nclusters, err, s);
}

cudaError_t device_error_word(int32_t **ptr) {
  return cudaGetSymbolAddress(reinterpret_cast<void **>(ptr), g_error_word);
}

size_t factor_smem_bytes(int nc, int ldt, size_t elem) {
  const size_t ncp = (size_t)((nc + 7) & ~7);
  // FP32 register-tile chains: the one-barrier job's two tail buffers and scalar sets, or
  // the compact-WY job's pivot column, Gram row and pivot rows; then the chain's R (the
  // compact-WY job's panel buffers come on top, f32wy_smem_extra_bytes)
  if (elem == sizeof(float))
    return sizeof(float) * (std::max((size_t)2 * kF32TileRows + 8, (size_t)kF32TileRows + 3 * ncp) +
                            (size_t)nc * (ncp + 1));
  return elem * ((size_t)nc * (size_t)ldt + 2 * ncp);
}

int factor_max_rows(int nc, int ctas_per_sm, size_t smem_per_sm, size_t reserved_per_block,
                    size_t optin_per_block, size_t elem) {
  if (ctas_per_sm < 1) return 0;
  size_t per_cta = smem_per_sm / (size_t)ctas_per_sm;
  if (per_cta <= reserved_per_block) return 0;
  per_cta -= reserved_per_block;
  if (per_cta > optin_per_block) per_cta = optin_per_block;
  const size_t extra = factor_smem_bytes(nc, 0, elem);
  if (per_cta <= extra) return 0;
  int rows = (int)((per_cta - extra) / (elem * (size_t)nc));
  return rows >= 16 ? (rows & ~15) : (rows & ~7);  // multiples of 16 keep the half-warps full
}

bool factor_tile_choice(int n, int nc, int leaf_h, size_t smem_per_sm, size_t reserved_per_block,
                        size_t optin_per_block, int max_cps, int &tile_h, int &cps) {
  for (int c = max_cps < 3 ? max_cps : 3; c >= 1; --c) {
    int rows = factor_max_rows(nc, c, smem_per_sm, reserved_per_block, optin_per_block);
    if (rows > 512) rows = 512;  // the apply kernels stage at most 512 rows per tile
    // a third CTA per SM pays only while its tile still holds two triangles' worth of rows
    const int need = (c >= 3) ? 2 * n : n;
    if (rows >= need && rows >= 8) {
      tile_h = rows < (leaf_h > n ? leaf_h : n) ? rows : (leaf_h > n ? leaf_h : n);
      cps = c;
      return true;
    }
  }
  return false;
}

cudaError_t launch_factor(const FactorParamsT<double> &p, int njobs, cudaStream_t s, int ctas_per_sm) {
  return launch_factor_any(p, njobs, ctas_per_sm, s);
}

cudaError_t launch_factor_batch(const BatchParams &p, int cmax, int grid, size_t smem_bytes, cudaStream_t s,
                                bool wy) {
  auto go = [&](auto kernel) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    kernel<<<grid, kThreads, smem_bytes, s>>>(p);
    return cudaGetLastError();
  };
  if (wy) {
    if (cmax <= 2) return go(k_factor_batch<2, true>);
    if (cmax <= 4) return go(k_factor_batch<4, true>);
    if (cmax <= 8) return go(k_factor_batch<8, true>);
    return go(k_factor_batch<16, true>);
  }
  if (cmax <= 1) return go(k_factor_batch<1, false>);
  if (cmax <= 2) return go(k_factor_batch<2, false>);
  if (cmax <= 4) return go(k_factor_batch<4, false>);
  if (cmax <= 8) return go(k_factor_batch<8, false>);
  return go(k_factor_batch<16, false>);
}

}  // namespace tsqr
