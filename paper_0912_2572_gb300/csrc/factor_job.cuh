// Device code of one factorization job, shared by the launch-per-level kernels and the
// persistent kernels (factor.cu, resident.cu): the FP64 shared-memory tile job (GEQRT /
// TSQRT / TTQRT tiles of paper §2.2-§2.3), the FP32 register-tile chain job of the mixed
// path, and the finishing step of a batched instance (R with diag >= 0, X by back
// substitution). The design notes of each job are beside it.
#pragma once
#include <cstdint>
#include <type_traits>

#include "tsqr_internal.h"
#include "warp_reduce.cuh"

namespace tsqr {
namespace {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

// One warp copies cnt doubles, 16 bytes per lane access when both addresses are 16-byte
// aligned (the caller's leading dimension decides), 8 bytes otherwise. LD loads one
// element or pair from the source (read-only input, or an L2 read of data another CTA of
// the same launch may have written).
template <typename LD1, typename LD2>
__device__ __forceinline__ void warp_copy(double *dst, const double *src, int cnt, int lane, LD1 ld1, LD2 ld2) {
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
    const int c2 = cnt >> 1;
    for (int i = lane; i < c2; i += 32) reinterpret_cast<double2 *>(dst)[i] = ld2(reinterpret_cast<const double2 *>(src) + i);
    if ((cnt & 1) && lane == 0) dst[cnt - 1] = ld1(src + cnt - 1);
  } else {
    for (int i = lane; i < cnt; i += 32) dst[i] = ld1(src + i);
  }
}

// Column slots. The FP64 job's column work is dealt to 14 worker half-warps (warps 0..6;
// warp 7 is the scalar warp): worker rank v (0..13) owns columns cs + v + 14 t. The rank
// of a warp rotates with the step, so the warp that takes the extra slot of an uneven
// step changes from step to step: a CTA's warp w always runs on SM sub-partition w mod 4,
// and with a fixed order the same sub-partition's FP64 pipe would carry the extra slots
// of every CTA on the SM.
constexpr int kColHalfWarps = 14;
constexpr int kWorkerWarps = kColHalfWarps / 2;

__host__ __device__ constexpr int job_nc_max(int cmax) { return cmax > 8 ? 144 : 16 * cmax; }
__host__ __device__ constexpr int job_slots_max(int cmax) {
  return (job_nc_max(cmax) + kColHalfWarps - 1) / kColHalfWarps;
}

// Gram row of step j: Pg[c] = sum_{i in [lo,hi)} T[j][i] T[c][i] for c = cs + v + 14 t
// (t < NS), v this half-warp's worker rank. The warp issues exactly its NS slots, so no
// predicated-off DFMA is issued; only half-warp 1 of the last slot can fall past nc.
template <int NS, typename R>
__device__ __forceinline__ void gram_row(const R *__restrict__ T, int ldt, int j, int cs, int nc, int lo,
                                         int hi, int v, int hl, R *__restrict__ Pg) {
  constexpr int C = pow2ceil(NS);
  const int cb = cs + v;
  R acc[C];
#pragma unroll
  for (int t = 0; t < C; ++t) acc[t] = R(0);
  const R *Tj = T + (size_t)j * ldt;
  for (int i = lo + hl; i < hi; i += 16) {
    const R x = Tj[i];
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int c = cb + kColHalfWarps * t;
      if (t < NS - 1 || c < nc) acc[t] = fma(x, T[(size_t)c * ldt + i], acc[t]);
    }
  }
  int idx;
  const R s = treduce16<C, R>(acc, hl, idx);
  const int c = cb + kColHalfWarps * idx;
  if ((hl & (16 / C - 1)) == 0 && idx < NS && c < nc) Pg[c] = s;
}

// Trailing update of step j: T[c][i] -= CF[c] * T[j][i] for c = cs + v + 14 t, i in [lo, hi).
template <int NS, typename R>
__device__ __forceinline__ void trailing_update(R *__restrict__ T, int ldt, int j, int cs, int nc, int lo,
                                                int hi, int v, int hl, const R *__restrict__ CF) {
  const int cb = cs + v;
  R cf[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    const int c = cb + kColHalfWarps * t;
    cf[t] = (c < nc) ? CF[c] : R(0);
  }
  const R *Tj = T + (size_t)j * ldt;
  for (int i = lo + hl; i < hi; i += 16) {
    const R x = Tj[i];
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int c = cb + kColHalfWarps * t;
      if (t < NS - 1 || c < nc) {
        R *q = T + (size_t)c * ldt + i;
        *q = fma(-cf[t], x, *q);
      }
    }
  }
}

// Slots of the worker warp of rank rw (its half-warps have ranks 2 rw and 2 rw + 1).
__device__ __forceinline__ int worker_slots(int cs, int nc, int rw) {
  const int r = nc - cs - 2 * rw;
  return r <= 0 ? 0 : (r + kColHalfWarps - 1) / kColHalfWarps;
}

// Runs OP<NS>(...) for the warp's exact slot count (1..11, at most job_slots_max(CMAX)).
#define TSQR_SLOT_CASES(OP, NSMAX, ARGS)                                                    \
  switch (ns) {                                                                           \
    case 1: OP<1, R> ARGS; return;                                                        \
    case 2: if (NSMAX >= 2) OP<(NSMAX >= 2 ? 2 : 1), R> ARGS; return;                    \
    case 3: if (NSMAX >= 3) OP<(NSMAX >= 3 ? 3 : 1), R> ARGS; return;                    \
    case 4: if (NSMAX >= 4) OP<(NSMAX >= 4 ? 4 : 1), R> ARGS; return;                    \
    case 5: if (NSMAX >= 5) OP<(NSMAX >= 5 ? 5 : 1), R> ARGS; return;                    \
    case 6: if (NSMAX >= 6) OP<(NSMAX >= 6 ? 6 : 1), R> ARGS; return;                    \
    case 7: if (NSMAX >= 7) OP<(NSMAX >= 7 ? 7 : 1), R> ARGS; return;                    \
    case 8: if (NSMAX >= 8) OP<(NSMAX >= 8 ? 8 : 1), R> ARGS; return;                    \
    case 9: if (NSMAX >= 9) OP<(NSMAX >= 9 ? 9 : 1), R> ARGS; return;                    \
    case 10: if (NSMAX >= 10) OP<(NSMAX >= 10 ? 10 : 1), R> ARGS; return;                \
    case 11: if (NSMAX >= 11) OP<(NSMAX >= 11 ? 11 : 1), R> ARGS; return;                \
    default: return;                                                                      \
  }

template <int CMAX, typename R>
__device__ __forceinline__ void gram_row_dispatch(const R *T, int ldt, int j, int cs, int nc, int lo, int hi,
                                                  int v, int hl, int rw, R *Pg) {
  constexpr int NM = job_slots_max(CMAX);
  const int ns = worker_slots(cs, nc, rw);
  TSQR_SLOT_CASES(gram_row, NM, (T, ldt, j, cs, nc, lo, hi, v, hl, Pg))
}

template <int CMAX, typename R>
__device__ __forceinline__ void update_dispatch(R *T, int ldt, int j, int cs, int nc, int lo, int hi, int v,
                                                int hl, int rw, const R *CF) {
  constexpr int NM = job_slots_max(CMAX);
  const int ns = worker_slots(cs, nc, rw);
  TSQR_SLOT_CASES(trailing_update, NM, (T, ldt, j, cs, nc, lo, hi, v, hl, CF))
}
#undef TSQR_SLOT_CASES

// Scalars of the reflector that maps x = [alpha; tail], ||tail||^2 = s2, onto beta e_1
// (Golub & Van Loan's sign choice, beta = -sign(alpha) ||x||, sign(0) = +1), in the form
// the kernel stores: v = [1; scale * tail], H = I - tau v v^T. With nrm = ||x||:
//   scale = sign(alpha) / (|alpha| + nrm),  tau = 1 + |alpha| / nrm,
//   tau * scale = sign(alpha) / nrm,
// which needs one reciprocal square root and one division. s2 == 0 gives H = I.
template <typename R>
struct Refl {
  R tau, scale, beta, ts;
};

__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }

template <typename R>
__device__ __forceinline__ Refl<R> reflector(R alpha, R s2) {
  Refl<R> r;
  if (s2 == R(0)) {
    r.tau = R(0);
    r.scale = R(0);
    r.beta = alpha;
    r.ts = R(0);
    return r;
  }
  const R s = fma(alpha, alpha, s2);
  const R rn = rsqrt_t(s);
  const R nrm = s * rn;
  const R sg = (alpha < R(0)) ? R(-1) : R(1);
  const R aa = fabs(alpha);
  r.beta = -sg * nrm;
  r.scale = sg / (aa + nrm);
  r.tau = fma(aa, rn, R(1));
  r.ts = sg * rn;
  return r;
}

// One FP64 job: the tiles of a chain or a tree node, run by the whole CTA (256 threads) in
// the shared-memory buffer smraw. Reads of V and B go through L2 (ld.global.cg): in the
// persistent batched kernel they may have been written by another CTA of the same launch.
//
// Warp 7 is the scalar warp. A step's reflector (the pivot column's norm, one rsqrt, one
// division) is a chain of about twenty dependent FP64 instructions, each waiting for the
// FP64 pipe behind the other warps' DFMA streams; run between the dot products and the
// update it took a quarter of every column step. Here the scalar warp computes the norm
// and the reflector *while* the worker warps compute the step's dot products, so only
// the two-deep coefficient step (w = p_k + scale g_k; coefficient ts w; new pivot entry
// p_k - tau w) separates the dot products from the update. The hand-offs are
// producer/consumer named barriers (bar.arrive / bar.sync); the end of the update is a
// full barrier (the next norm and dot products read column j + 1).
constexpr int kScalarWarp = kWorkerWarps;
static_assert(kThreads == 32 * (kWorkerWarps + 1), "seven worker warps and the scalar warp");

__device__ __forceinline__ void bar_sync_n(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive_n(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// EARLY_PF: the scalar warp loads the next pivot row at the start of the step (its L2
// latency overlaps the norm and the reflector, which matters on tree nodes, where the
// update is short) instead of after the coefficients (fewer live registers: the batched
// kernel, at its register cap, keeps that order).
//
// COH: inputs and descriptors are read through L2 only (the resident kernel, whose inputs
// and tables change while it runs); otherwise A goes through the read-only cache.
template <int CMAX, bool EARLY_PF, bool COH = false>
__device__ __forceinline__ void run_job(const FactorParamsT<double> &p, const JobDesc job, unsigned char *smraw) {
  using R = double;
  R *sm = reinterpret_cast<R *>(smraw);
  const int n = p.n, nc = p.nc, ldt = p.ldt;
  const int ncp = (nc + 7) & ~7;
  R *T = sm;                            // tile, column-major, nc columns of ldt rows
  R *PC = T + (size_t)nc * ldt;         // the step's dot products (workers -> scalar warp),
                                        // turned in place into update coefficients
  R *PV = PC + ncp;                     // staged pivot row (TSQRT / TTQRT; scalar warp only)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool sw = (warp == kScalarWarp);
  const int hl = tid & 15, hsub = (tid >> 4) & 1;
  const int64_t pr = job.piv_row;
  auto piv_ptr = [&](int j, int c) -> R * {
    return (c < n) ? p.V + pr + j + (int64_t)c * p.ldv : p.B + pr + j + (int64_t)(c - n) * p.ldb;
  };
  constexpr int PCN = (job_nc_max(CMAX) + 31) / 32;  // columns after the pivot, per lane
  TSQR_CHECK_OR_SKIP(pr >= 0 && (p.rows == 0 || pr + n <= p.rows) && job.tile_begin >= 0 &&
                         (p.ntiles == 0 || job.tile_begin + job.tile_count <= p.ntiles) && nc <= job_nc_max(CMAX),
                     p.err)

  for (int tt = 0; tt < job.tile_count; ++tt) {
    const TileDesc td = load_tile<COH>(p.tiles + job.tile_begin + tt);
    const int ht = td.nrows, kind = td.kind, off = td.off;
    const int64_t r0 = td.row0;
    TSQR_CHECK_OR_SKIP(r0 >= 0 && ht >= 1 && ht <= ldt && (p.rows == 0 || r0 + ht <= p.rows) && kind >= GEQRT &&
                           kind <= TTQRT && off >= 0 && off < n && td.refl >= 0 &&
                           (p.nrefl == 0 || td.refl + n <= p.nrefl),
                       p.err)
    const bool ge = (kind == GEQRT);
    // a TTQRT piece starting at row `off` of the child is untouched by reflectors j < off
    const int j0 = (kind == TTQRT) ? off : 0;

    // stage the tile: GEQRT/TSQRT tiles come from A (first touch), TTQRT from V
    for (int c = warp; c < nc; c += kThreads / 32) {
      R *dst = T + (size_t)c * ldt;
      if (c < n && kind != TTQRT) {
        const double *src = p.A + r0 + (int64_t)c * p.lda;
        warp_copy(dst, src, ht, lane, [](const double *q) { return ld_input<COH>(q); },
                  [](const double2 *q) { return ld_input<COH>(q); });
      } else {
        const R *src = (c < n) ? p.V + r0 + (int64_t)c * p.ldv : p.B + r0 + (int64_t)(c - n) * p.ldb;
        warp_copy(dst, src, ht, lane, [](const double *q) { return __ldcg(q); },
                  [](const double2 *q) { return __ldcg(q); });
      }
    }
    if (!ge)
      for (int c = tid; c < nc; c += kThreads) PV[c] = (c >= j0) ? __ldcg(piv_ptr(j0, c)) : R(0);
    for (int j = tid; j < j0; j += kThreads) {  // identity reflectors
      p.tau[td.refl + j] = R(0);
      p.scl[td.refl + j] = R(0);
    }
    __syncthreads();

    for (int j = j0; j < n; ++j) {
      int lo, hi;
      refl_rows(kind, j, ht, lo, hi, off);
      if (!sw) {
        const int rw = (warp + j) % kWorkerWarps;  // this step's worker rank
        const int v = 2 * rw + hsub;
        gram_row_dispatch<CMAX, R>(T, ldt, j, j + 1, nc, lo, hi, v, hl, rw, PC);
        bar_arrive_n(1, kThreads);
        bar_sync_n(2, kThreads);
        update_dispatch<CMAX, R>(T, ldt, j, j + 1, nc, lo, hi, v, hl, rw, PC);
      } else {
        // the next pivot row (not written before step j+1) is loaded now, so its L2 latency
        // overlaps this step's norm and reflector
        R pf[PCN];
        const bool do_pf = !ge && j + 1 < n;
        if (EARLY_PF && do_pf) {
#pragma unroll
          for (int q = 0; q < PCN; ++q) {
            const int c = j + 1 + lane + 32 * q;
            pf[q] = (c < nc) ? __ldcg(piv_ptr(j + 1, c)) : R(0);
          }
        }
        // squared norm of the pivot column's tail (two partial sums per lane), then the reflector
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
        const Refl<R> rf = reflector<R>(ge ? Tj[j] : PV[j], s2);
        bar_sync_n(1, kThreads);  // the workers' dot products are in PC
        R pk[PCN];
#pragma unroll
        for (int q = 0; q < PCN; ++q) {
          const int c = j + 1 + lane + 32 * q;
          if (c < nc) {
            const R p0 = ge ? T[(size_t)c * ldt + j] : PV[c];
            const R w = fma(rf.scale, PC[c], p0);
            PC[c] = rf.ts * w;
            pk[q] = fma(-rf.tau, w, p0);
          }
        }
        bar_arrive_n(2, kThreads);  // the coefficients are in PC
        // the new pivot row and the reflector's scalars, then the next pivot row's staging
        // (PV[c] for c > j was read above by this same lane)
#pragma unroll
        for (int q = 0; q < PCN; ++q) {
          const int c = j + 1 + lane + 32 * q;
          if (c < nc) {
            if (ge)
              T[(size_t)c * ldt + j] = pk[q];
            else
              *piv_ptr(j, c) = pk[q];
          }
        }
        if (lane == 0) {
          if (ge)
            T[(size_t)j * ldt + j] = rf.beta;
          else
            *piv_ptr(j, j) = rf.beta;
          p.tau[td.refl + j] = rf.tau;
          p.scl[td.refl + j] = rf.scale;
        }
        if (do_pf) {
#pragma unroll
          for (int q = 0; q < PCN; ++q) {
            const int c = j + 1 + lane + 32 * q;
            if (c < nc) PV[c] = EARLY_PF ? pf[q] : __ldcg(piv_ptr(j + 1, c));
          }
        }
        __syncwarp();
      }
      __syncthreads();
    }

    // write the tile back: GEQRT -> R above / V below the diagonal, TSQRT -> dense
    // reflector tails, TTQRT -> the upper triangle only (the child's own leaf
    // reflectors live below its diagonal)
    for (int c = warp; c < nc; c += kThreads / 32) {
      R *dst = (c < n) ? p.V + r0 + (int64_t)c * p.ldv : p.B + r0 + (int64_t)(c - n) * p.ldb;
      const R *src = T + (size_t)c * ldt;
      const int lim = (kind == TTQRT && c < n) ? max(0, min(ht, c + 1 - off)) : ht;
      warp_copy(dst, src, lim, lane, [](const double *q) { return *q; }, [](const double2 *q) { return *q; });
    }
    __syncthreads();
  }
}

// ------------------------------------------------------ FP32 chains: register tiles
// The FP32 chains of the mixed path keep their tile in registers. On the FP32 pipe the
// shared-memory tile of the kernel above is bound by instruction issue (an address
// computation and a shared-memory access per FMA) and a column step lasts a fraction of
// a microsecond, so nothing on a step's critical path may go to L2. Here:
//   * thread (hw, hl) holds columns hw + 16 t (t < CPT) of rows hl + 16 r (r < kF32Rpt)
//     of a 128-row tile; a column step moves only the pivot column j (the reflector's
//     tail) and the step's scalars through shared memory, and the Gram row and the
//     rank-1 update are register FMAs over the columns still active;
//   * the chain's R (its n pivot rows, n x nc) stays in shared memory for the whole chain:
//     the leaf's first tile leaves it there, each triangle-on-tile step reads and
//     rewrites its pivot row there, and R goes to global memory once, at the end;
//   * the slot range of a step is the same for the two half-warps of a warp (their
//     shuffles must match); a boundary slot is guarded per half-warp.
template <int CPT, int T0>
__device__ __forceinline__ void f32_gram(const float (&v)[CPT][kF32Rpt], const float (&x)[kF32Rpt], int j, int hw,
                                         int hl, int nc, float *Pg) {
  constexpr int NA = CPT - T0;
  constexpr int C = pow2ceil(NA);
  float acc[C];
#pragma unroll
  for (int t = 0; t < C; ++t) acc[t] = 0.f;
#pragma unroll
  for (int t = 0; t < NA; ++t)
#pragma unroll
    for (int r = 0; r < kF32Rpt; ++r) acc[t] = fmaf(x[r], v[T0 + t][r], acc[t]);
  int idx;
  const float s = treduce16<C, float>(acc, hl, idx);
  const int c = hw + 16 * (T0 + idx);
  if ((hl & (16 / C - 1)) == 0 && idx < NA && c >= j && c < nc) Pg[c] = s;
}

template <int CPT, int T0>
__device__ __forceinline__ void f32_update(float (&v)[CPT][kF32Rpt], const float (&x)[kF32Rpt], int j, int hw,
                                           int nc, const float *CF) {
#pragma unroll
  for (int t = T0; t < CPT; ++t) {
    const int c = hw + 16 * t;
    if (c <= j || c >= nc) continue;  // the first slot may hold column j or an earlier one
    const float cf = CF[c];
#pragma unroll
    for (int r = 0; r < kF32Rpt; ++r) v[t][r] = fmaf(-cf, x[r], v[t][r]);
  }
}

template <int CPT>
__device__ __forceinline__ void f32_gram_dispatch(const float (&v)[CPT][kF32Rpt], const float (&x)[kF32Rpt], int j,
                                                  int t0, int hw, int hl, int nc, float *Pg) {
  switch (t0) {
    case 0: f32_gram<CPT, 0>(v, x, j, hw, hl, nc, Pg); return;
#define TSQR_F32_GRAM(T) \
    case T: if (CPT > T) f32_gram<CPT, (CPT > T ? T : 0)>(v, x, j, hw, hl, nc, Pg); return;
    TSQR_F32_GRAM(1) TSQR_F32_GRAM(2) TSQR_F32_GRAM(3) TSQR_F32_GRAM(4) TSQR_F32_GRAM(5) TSQR_F32_GRAM(6)
    TSQR_F32_GRAM(7)
#undef TSQR_F32_GRAM
    default: return;
  }
}

template <int CPT>
__device__ __forceinline__ void f32_update_dispatch(float (&v)[CPT][kF32Rpt], const float (&x)[kF32Rpt], int j,
                                                    int t0, int hw, int nc, const float *CF) {
  switch (t0) {
    case 0: f32_update<CPT, 0>(v, x, j, hw, nc, CF); return;
#define TSQR_F32_UPD(T) \
    case T: if (CPT > T) f32_update<CPT, (CPT > T ? T : 0)>(v, x, j, hw, nc, CF); return;
    TSQR_F32_UPD(1) TSQR_F32_UPD(2) TSQR_F32_UPD(3) TSQR_F32_UPD(4) TSQR_F32_UPD(5) TSQR_F32_UPD(6)
    TSQR_F32_UPD(7)
#undef TSQR_F32_UPD
    default: return;
  }
}

// One chain job (a leaf's GEQRT tile, then TSQRT tiles; at most 16 * CPT columns) with
// register tiles. Shared memory: the pivot column (kF32TileRows), the Gram row (ncp),
// two pivot-row buffers for the leaf tile (2 ncp) and the chain's R (n rows of ncp + 1).
template <int CPT, bool COH = false>
__device__ __forceinline__ void run_job_f32r(const FactorParamsT<float> &p, const JobDesc job, unsigned char *smraw) {
  float *sm = reinterpret_cast<float *>(smraw);
  const int n = p.n, nc = p.nc;
  const int ncp = (nc + 7) & ~7;
  float *xcol = sm;
  float *PC = xcol + kF32TileRows;
  float *PVb = PC + ncp;
  const int ldr = ncp + 1;    // odd: the end-of-chain column walk is conflict-free
  float *Rs = PVb + 2 * ncp;  // R(i, c) at Rs[i * ldr + c]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int hw = tid >> 4, hl = tid & 15;
  const int hw_hi = 2 * warp + 1;  // the larger column offset of the warp's half-warps
  const int64_t pr = job.piv_row;
  float v[CPT][kF32Rpt];

  for (int tt = 0; tt < job.tile_count; ++tt) {
    const TileDesc td = load_tile<COH>(p.tiles + job.tile_begin + tt);
    const int ht = td.nrows;
    const int64_t r0 = td.row0;
    const bool ge = (td.kind == GEQRT);
    // load the tile (A is FP64, rounded here); rows past ht and columns past nc are 0
#pragma unroll
    for (int t = 0; t < CPT; ++t) {
      const int c = hw + 16 * t;
#pragma unroll
      for (int r = 0; r < kF32Rpt; ++r) {
        const int i = hl + 16 * r;
        float val = 0.f;
        if (c < nc && i < ht)
          val = (c < n) ? (float)ld_input<COH>(p.A + r0 + i + (int64_t)c * p.lda)
                        : __ldcg(p.B + r0 + i + (int64_t)(c - n) * p.ldb);
        v[t][r] = val;
      }
    }
    __syncthreads();

    for (int j = 0; j < n; ++j) {
      const int tj = j >> 4, jl = j & 15;
      float *PV = ge ? PVb + (j & 1) * ncp : Rs + j * ldr;
      // (A) publish the pivot column (its owner half-warp) and, for the leaf tile, the
      //     pivot row (its owner lane in every half-warp)
      if (hw == jl) {
#pragma unroll
        for (int t = 0; t < CPT; ++t)
          if (t == tj)
#pragma unroll
            for (int r = 0; r < kF32Rpt; ++r) xcol[hl + 16 * r] = v[t][r];
      }
      if (ge && hl == jl) {
#pragma unroll
        for (int r = 0; r < kF32Rpt; ++r)
          if (r == tj)
#pragma unroll
            for (int t = 0; t < CPT; ++t) {
              const int c = hw + 16 * t;
              if (c >= j && c < nc) PV[c] = v[t][r];
            }
      }
      __syncthreads();
      // (B) the tail of column j on this lane's rows, then the Gram row
      float x[kF32Rpt];
#pragma unroll
      for (int r = 0; r < kF32Rpt; ++r) {
        const int i = hl + 16 * r;
        x[r] = (ge && i <= j) ? 0.f : xcol[i];
      }
      {
        const int d = j - hw_hi;
        f32_gram_dispatch<CPT>(v, x, j, d <= 0 ? 0 : (d + 15) >> 4, hw, hl, nc, PC);
      }
      __syncthreads();
      // (C) warp 0: the reflector's scalars, the update coefficients and the new pivot row.
      //     Up to 64 columns all loads go first (the columns are independent, and stores
      //     between loads would serialize them: about 6% faster chains at n <= 64); at 128
      //     columns the extra live registers cost more than that.
      if (warp == 0) {
        const Refl<float> rf = reflector<float>(PV[j], PC[j]);
        if constexpr (CPT <= 4) {
          constexpr int QN = (16 * CPT + 31) / 32;
          float pk[QN], g[QN];
#pragma unroll
          for (int q = 0; q < QN; ++q) {
            const int c = j + 1 + lane + 32 * q;
            pk[q] = (c < nc) ? PV[c] : 0.f;
            g[q] = (c < nc) ? PC[c] : 0.f;
          }
#pragma unroll
          for (int q = 0; q < QN; ++q) {
            const int c = j + 1 + lane + 32 * q;
            const float w = fmaf(rf.scale, g[q], pk[q]);
            if (c < nc) {
              PC[c] = rf.ts * w;
              PV[c] = fmaf(-rf.tau, w, pk[q]);
            }
          }
        } else {
          for (int c = j + 1 + lane; c < nc; c += 32) {
            const float pk = PV[c];
            const float w = fmaf(rf.scale, PC[c], pk);
            PC[c] = rf.ts * w;
            PV[c] = fmaf(-rf.tau, w, pk);
          }
        }
        if (lane == 0) {
          PV[j] = rf.beta;
          p.tau[td.refl + j] = rf.tau;
          p.scl[td.refl + j] = rf.scale;
        }
      }
      __syncthreads();
      // (D) the rank-1 update; on the leaf tile the owner lane of row j takes the new row
      {
        const int d = j + 1 - hw_hi;
        f32_update_dispatch<CPT>(v, x, j, d <= 0 ? 0 : (d + 15) >> 4, hw, nc, PC);
      }
      if (ge && hl == jl) {
#pragma unroll
        for (int r = 0; r < kF32Rpt; ++r)
          if (r == tj)
#pragma unroll
            for (int t = 0; t < CPT; ++t) {
              const int c = hw + 16 * t;
              if (c >= j && c < nc) v[t][r] = PV[c];
            }
      }
    }
    __syncthreads();
    // the leaf tile's R (rows < n, upper part; right-hand-side columns in full) becomes
    // the chain's R in shared memory
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
    // write the tile back: the leaf tile holds R above and reflectors below the diagonal
    // (R is rewritten from shared memory at the end), a TSQRT tile dense reflector tails
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
  // the chain's R to its pivot rows in global memory
  for (int e = tid; e < n * nc; e += kThreads) {
    const int i = e % n, c = e / n;
    if (i <= c || c >= n) {
      float *dst = (c < n) ? p.V + pr + i + (int64_t)c * p.ldv : p.B + pr + i + (int64_t)(c - n) * p.ldb;
      *dst = Rs[i * ldr + c];
    }
  }
  __syncthreads();
}

// Finishing an instance: R out with diag >= 0, and X = R^{-1} (Q^T B)[0:n] when the
// right-hand sides were factored along (back substitution in shared memory).
__device__ __forceinline__ void finish_instance(const BatchInst &in, int64_t row64, unsigned char *smraw) {
  const int n = in.n, k = in.k;
  const double *Rr = in.V64 + row64;  // R(i, j) = Rr[i + j * ldv64]
  if (in.R) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e % n, j = e / n;
      const double di = (__ldcg(Rr + i + (int64_t)i * in.ldv64) < 0.0) ? -1.0 : 1.0;
      in.R[i + (int64_t)j * in.ldr] = (i <= j) ? di * __ldcg(Rr + i + (int64_t)j * in.ldv64) : 0.0;
    }
  }
  if (k > 0 && in.X) {
    double *xs = reinterpret_cast<double *>(smraw);  // n * k
    const double *C = in.B + row64;                   // (Q^T B)[0:n] in the pivot rows
    for (int e = threadIdx.x; e < n * k; e += blockDim.x) {
      const int i = e % n, c = e / n;
      xs[e] = __ldcg(C + i + (int64_t)c * in.ldb);
    }
    __syncthreads();
    for (int i = n - 1; i >= 0; --i) {
      const double rii = __ldcg(Rr + i + (int64_t)i * in.ldv64);
      for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if (rii == 0.0) {
          if (in.status) atomicExch(in.status, 4);
          xs[i + c * n] = 0.0;
        } else {
          xs[i + c * n] /= rii;
        }
      }
      __syncthreads();
      for (int e = threadIdx.x; e < i * k; e += blockDim.x) {
        const int l = e % i, c = e / i;
        xs[l + c * n] = fma(-__ldcg(Rr + l + (int64_t)i * in.ldv64), xs[i + c * n], xs[l + c * n]);
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < n * k; e += blockDim.x) {
      const int i = e % n, c = e / n;
      in.X[i + (int64_t)c * in.ldx] = xs[e];
    }
  }
  __syncthreads();
}

}  // namespace
}  // namespace tsqr
