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
// update is short) instead of after the coefficients (fewer live registers: the resident
// kernel, at its register cap, keeps that order). The row is not written before step j+1,
// so both orders load the same values and give bitwise the same results.
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
//     shuffles must match); a boundary slot is guarded per half-warp;
//   * one block barrier per column step. Every half-warp owns whole columns, so it needs
//     nobody else's results to finish a step on them: it reduces its own Gram entries over
//     its 16 lanes, computes its own coefficients and new pivot-row entries, and updates
//     its own columns. Only the reflector crosses half-warps: the owner of column j + 1,
//     once that column is updated, computes reflector j + 1 (tail norm, one rsqrt, one
//     division) and publishes its tail and scalars, which the step's barrier makes
//     visible. Tail and scalars are double-buffered by step parity (a buffer is rewritten
//     only after the next barrier, when every reader is done with it). An earlier form of
//     the job published the pivot column (barrier), reduced the Gram row into shared
//     memory (barrier), let warp 0 turn it into coefficients (barrier) and then updated:
//     bound by those hand-offs, not by its FMAs, it took about 2,700 cycles per step at
//     n = 128 with one CTA per SM and 3,300 with two, against 1,950 and 2,500 here.

// Lowest lane holding the total of value i after treduce16<C> (the total is replicated on
// the 16 / C lanes above it).
template <int C>
__device__ __forceinline__ int treduce16_lane(int i) {
  int l = 0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int half = (C >> s) >> 1;
    if (half >= 1 && (i & half)) l |= (8 >> s);
  }
  return l;
}

// Register element v[t][r] with a runtime r (an unrolled select keeps v in registers).
template <int CPT>
__device__ __forceinline__ float f32s_get(const float (&v)[CPT][kF32Rpt], int t, int r) {
  float out = 0.f;
#pragma unroll
  for (int tt = 0; tt < CPT; ++tt)
#pragma unroll
    for (int rr = 0; rr < kF32Rpt; ++rr)
      if (tt == t && rr == r) out = v[tt][rr];
  return out;
}
template <int CPT>
__device__ __forceinline__ void f32s_set(float (&v)[CPT][kF32Rpt], int t, int r, float x) {
#pragma unroll
  for (int tt = 0; tt < CPT; ++tt)
#pragma unroll
    for (int rr = 0; rr < kF32Rpt; ++rr)
      if (tt == t && rr == r) v[tt][rr] = x;
}

// Step j for this warp's NA highest column slots (t = CPT - NA .. CPT - 1; the lower slots
// hold only columns <= j). x: the tail of pivot column j on this lane's rows; Rs: the chain's
// R (row j is the pivot row of a triangle-on-tile step); for the leaf tile (GE) the pivot row
// is the tile's own row j, which lane j mod 16 of each half-warp holds. pub(column) publishes
// reflector j+1 from the registers of slot T0 (its owner half-warp only).
template <int CPT, int NA, bool GE, typename PUB>
__device__ __forceinline__ void f32s_step(float (&v)[CPT][kF32Rpt], const float (&x)[kF32Rpt], int j, int nc,
                                          int hw, int hl, float *Rs, int ldr, float tau, float scale, float ts,
                                          PUB &pub) {
  constexpr int T0 = CPT - NA;
  constexpr int C = pow2ceil(NA);
  const int lane = threadIdx.x & 31;
  float g[C];
#pragma unroll
  for (int i = 0; i < C; ++i) g[i] = 0.f;
#pragma unroll
  for (int i = 0; i < NA; ++i)
#pragma unroll
    for (int r = 0; r < kF32Rpt; ++r) g[i] = fmaf(x[r], v[T0 + i][r], g[i]);
  int idx;
  const float gt = treduce16<C, float>(g, hl, idx);
  const int c_me = hw + 16 * (T0 + idx);
  const bool ok = idx < NA && c_me > j && c_me < nc;
  if constexpr (GE) {  // the leaf tile's pivot row j goes to Rs, where every lane of the half-warp reads it
    if (hl == (j & 15))
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        const int c = hw + 16 * (T0 + i);
        if (c > j && c < nc) Rs[j * ldr + c] = f32s_get<CPT>(v, T0 + i, j >> 4);
      }
    __syncwarp();
  }
  float cf_me = 0.f, pk = 0.f;
  if (ok) {
    const float p0 = Rs[j * ldr + c_me];
    const float w = fmaf(scale, gt, p0);
    cf_me = ts * w;
    pk = fmaf(-tau, w, p0);
  }
  __syncwarp();  // every replica has read p0 before one of them overwrites it
  if (ok && (hl & (16 / C - 1)) == 0) Rs[j * ldr + c_me] = pk;
  if constexpr (GE) {  // the new pivot row back into the registers of its lane
    __syncwarp();
    if (hl == (j & 15))
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        const int c = hw + 16 * (T0 + i);
        if (c > j && c < nc) f32s_set<CPT>(v, T0 + i, j >> 4, Rs[j * ldr + c]);
      }
  }
  // the rank-1 update, slot T0 first: column j + 1 is always in its owner warp's lowest
  // active slot, so reflector j + 1 is published before the other slots are updated. A
  // slot's coefficient comes from the lane that reduced it.
#pragma unroll
  for (int i = 0; i < NA; ++i) {
    const float cf = __shfl_sync(0xffffffffu, cf_me, (lane & 16) + treduce16_lane<C>(i));
#pragma unroll
    for (int r = 0; r < kF32Rpt; ++r) v[T0 + i][r] = fmaf(-cf, x[r], v[T0 + i][r]);
    if (i == 0) pub(v[T0]);
  }
}

template <int CPT, bool GE, typename PUB>
__device__ __forceinline__ void f32s_dispatch(int na, float (&v)[CPT][kF32Rpt], const float (&x)[kF32Rpt], int j,
                                              int nc, int hw, int hl, float *Rs, int ldr, float tau, float scale,
                                              float ts, PUB &pub) {
  switch (na) {
#define TSQR_F32S_CASE(NA)                                                                      \
    case NA:                                                                                    \
      if constexpr (CPT >= NA) f32s_step<CPT, NA, GE>(v, x, j, nc, hw, hl, Rs, ldr, tau, scale, ts, pub); \
      return;
    TSQR_F32S_CASE(1) TSQR_F32S_CASE(2) TSQR_F32S_CASE(3) TSQR_F32S_CASE(4)
    TSQR_F32S_CASE(5) TSQR_F32S_CASE(6) TSQR_F32S_CASE(7) TSQR_F32S_CASE(8)
#undef TSQR_F32S_CASE
    default: return;  // no column after j in this warp (never the owner of column j + 1)
  }
}

// One chain job with register tiles and one barrier per column step. Shared memory: two
// pivot-tail buffers (2 kF32TileRows), two scalar sets (8) and the chain's R (n rows of
// ncp + 1), within factor_smem_bytes(nc, ., 4).
template <int CPT, bool COH = false>
__device__ __forceinline__ void run_job_f32s(const FactorParamsT<float> &p, const JobDesc job, unsigned char *smraw) {
  float *sm = reinterpret_cast<float *>(smraw);
  const int n = p.n, nc = p.nc;
  const int ncp = (nc + 7) & ~7;
  const int ldr = ncp + 1;    // odd: the end-of-chain column walk is conflict-free
  float *xb = sm;             // tails of pivot columns j (buffer j mod 2)
  float *sb = xb + 2 * kF32TileRows;  // tau, scale, tau * scale of reflector j (buffer j mod 2)
  float *Rs = sb + 8;         // R(i, c) at Rs[i * ldr + c]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int hw = tid >> 4, hl = tid & 15;
  const int hw_hi = 2 * warp + 1;  // the larger column offset of the warp's half-warps
  const unsigned hmask = 0xffffu << (lane & 16);
  const int64_t pr = job.piv_row;
  float v[CPT][kF32Rpt];

  for (int tt = 0; tt < job.tile_count; ++tt) {
    const TileDesc td = load_tile<COH>(p.tiles + job.tile_begin + tt);
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
          val = (c < n) ? (float)ld_input<COH>(p.A + r0 + i + (int64_t)c * p.lda)
                        : __ldcg(p.B + r0 + i + (int64_t)(c - n) * p.ldb);
        v[t][r] = val;
      }
    }
    __syncthreads();  // the previous tile's readers of the buffers are done

    // reflector jn (column jn's owner half-warp, given the registers of column jn): its
    // tail, norm and scalars, published
    int jn = 0;
    auto pub = [&](float (&w)[kF32Rpt]) {
      if (jn >= n || hw != (jn & 15)) return;
      const int b = jn & 1, rn = jn >> 4;
      // the tail (rows below the pivot of a leaf tile, all rows of a tile under a
      // triangle) goes out as it is summed
      float s2 = 0.f, wn = 0.f;
#pragma unroll
      for (int r = 0; r < kF32Rpt; ++r) {
        float val = w[r];
        if (r == rn) wn = val;
        if (ge && hl + 16 * r <= jn) val = 0.f;
        s2 = fmaf(val, val, s2);
        xb[b * kF32TileRows + hl + 16 * r] = val;
      }
      const float alpha = ge ? __shfl_sync(hmask, wn, (lane & 16) + (jn & 15)) : Rs[jn * ldr + jn];
#pragma unroll
      for (int m = 8; m >= 1; m >>= 1) s2 += __shfl_xor_sync(hmask, s2, m);
      const Refl<float> rf = reflector<float>(alpha, s2);
      if (hl == 0) {
        sb[4 * b] = rf.tau;
        sb[4 * b + 1] = rf.scale;
        sb[4 * b + 2] = rf.ts;
        p.tau[td.refl + jn] = rf.tau;
        p.scl[td.refl + jn] = rf.scale;
        if (!ge) Rs[jn * ldr + jn] = rf.beta;
      }
      if (ge && hl == (jn & 15))
#pragma unroll
        for (int r = 0; r < kF32Rpt; ++r)
          if (r == rn) w[r] = rf.beta;
    };
    pub(v[0]);
    __syncthreads();

    for (int j = 0; j < n; ++j) {
      const int b = j & 1;
      float x[kF32Rpt];
#pragma unroll
      for (int r = 0; r < kF32Rpt; ++r) x[r] = xb[b * kF32TileRows + hl + 16 * r];
      const float tau = sb[4 * b], scale = sb[4 * b + 1], ts = sb[4 * b + 2];
      jn = j + 1;
      const int d = j - hw_hi;
      const int na = CPT - (d < 0 ? 0 : (d >> 4) + 1);
      if (ge)
        f32s_dispatch<CPT, true>(na, v, x, j, nc, hw, hl, Rs, ldr, tau, scale, ts, pub);
      else
        f32s_dispatch<CPT, false>(na, v, x, j, nc, hw, hl, Rs, ldr, tau, scale, ts, pub);
      __syncthreads();
    }
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
