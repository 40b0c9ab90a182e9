// Application of the TSQR orthogonal factor (sm_103a): B <- Q^T B, B <- Q B, and the
// thin Q = Q [I_n; 0] (paper §4, Table 2: Q costs what R costs; Property 1).
//
// The factor set is a list of launches of jobs; each job walks its tiles and each tile
// holds n reflectors v = [1 at pivot row j; scale_j * tail_j] (tsqr_internal.h). Q^T
// applies jobs launch by launch, tiles and reflectors in factorization order; Q applies
// everything in reverse.
//
// Two kernels:
//   * k_apply_warp: one warp per job, for B with at most 8 columns, and for forming a
//     thin Q of up to 32 columns in passes of 4. Each reflector is a dot product over the
//     tile rows, one warp-level transpose-reduce, and an update; no block barrier is
//     needed. With 4 columns a job stages 16.6 KB of a 512-row tile, so three CTAs of four
//     jobs fit per SM, and the independent jobs of a sub-partition's three warps hide one
//     another's reduction and shared-memory latency.
//   * k_apply_tile: one CTA per job and per pass of up to 64 columns, the structure of
//     the factor kernel. Used for many right-hand sides and for forming Q. When forming
//     Q every pivot-row block stays upper triangular (the root starts from
//     diag(sign(r_jj)) and each node's Q blocks are triangular), so reflector j only
//     touches columns >= j and forming Q costs as many flops as the factorization, not
//     twice as many.
#include "cluster_sync.cuh"
#include "tsqr_internal.h"
#include "warp_reduce.cuh"

namespace tsqr {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Runs BODY(r) for r = ra-1 down to 0 (ra <= 32, warp-uniform) through a fall-through
// switch: only the row slots the reflector needs are issued (a predicated-off FP64
// instruction still occupies the FP64 pipe), while r stays a compile-time register index.
#define TSQR_ROW_SLOTS(ra, RM, BODY)                                                        \
  switch ((ra) > (RM) ? (RM) : (ra)) {                                                      \
    case 32: if (RM >= 32) BODY(31)                                                         \
    case 31: if (RM >= 31) BODY(30)                                                         \
    case 30: if (RM >= 30) BODY(29)                                                         \
    case 29: if (RM >= 29) BODY(28)                                                         \
    case 28: if (RM >= 28) BODY(27)                                                         \
    case 27: if (RM >= 27) BODY(26)                                                         \
    case 26: if (RM >= 26) BODY(25)                                                         \
    case 25: if (RM >= 25) BODY(24)                                                         \
    case 24: if (RM >= 24) BODY(23)                                                         \
    case 23: if (RM >= 23) BODY(22)                                                         \
    case 22: if (RM >= 22) BODY(21)                                                         \
    case 21: if (RM >= 21) BODY(20)                                                         \
    case 20: if (RM >= 20) BODY(19)                                                         \
    case 19: if (RM >= 19) BODY(18)                                                         \
    case 18: if (RM >= 18) BODY(17)                                                         \
    case 17: if (RM >= 17) BODY(16)                                                         \
    case 16: if (RM >= 16) BODY(15)                                                         \
    case 15: if (RM >= 15) BODY(14)                                                         \
    case 14: if (RM >= 14) BODY(13)                                                         \
    case 13: if (RM >= 13) BODY(12)                                                         \
    case 12: if (RM >= 12) BODY(11)                                                         \
    case 11: if (RM >= 11) BODY(10)                                                         \
    case 10: if (RM >= 10) BODY(9)                                                          \
    case 9: if (RM >= 9) BODY(8)                                                            \
    case 8: if (RM >= 8) BODY(7)                                                            \
    case 7: if (RM >= 7) BODY(6)                                                            \
    case 6: if (RM >= 6) BODY(5)                                                            \
    case 5: if (RM >= 5) BODY(4)                                                            \
    case 4: if (RM >= 4) BODY(3)                                                            \
    case 3: if (RM >= 3) BODY(2)                                                            \
    case 2: if (RM >= 2) BODY(1)                                                            \
    case 1: BODY(0)                                                                         \
    default: break;                                                                         \
  }

// ------------------------------------------------------------- one warp per job
// One reflector (pivot row j, tail xv over rows [lo, hi), tau, scale) applied to the NA
// columns c0 .. c0 + NA - 1 of the warp's staged tile: dot products, one transpose-
// reduce, the pivot-row update, then the tail update. NA is exact, so no column that the
// reflector leaves unchanged issues an FMA (forming Q: reflector j touches columns >= j).
template <int NA, int RW, typename R>
__device__ __forceinline__ void warp_reflector(R *Bt, R *PR, int ldt, int n, int c0, bool ge, int j, int lo,
                                               int hi, int lane, const R (&xv)[RW], R tau, R sc) {
  constexpr int KP = pow2ceil(NA);
  R part[KP];
#pragma unroll
  for (int a = 0; a < KP; ++a) part[a] = R(0);
  R *Bc = Bt + (size_t)c0 * ldt;
  const int ra = (hi - lo + 31) >> 5;
#define TSQR_WDOT(r)                                                                        \
  {                                                                                         \
    const int i = lo + lane + 32 * (r);                                                     \
    if (i < hi) {                                                                           \
      _Pragma("unroll") for (int a = 0; a < NA; ++a) part[a] = fma(xv[r], Bc[a * ldt + i], part[a]); \
    }                                                                                       \
  }
  TSQR_ROW_SLOTS(ra, RW, TSQR_WDOT)
#undef TSQR_WDOT
  int idx;
  const R tot = treduce32<KP, R>(part, lane, idx);
  R cfv = R(0);
  if ((lane & (32 / KP - 1)) == 0 && idx < NA) {
    const int c = c0 + idx;
    R *pp = ge ? &Bt[c * ldt + j] : &PR[c * n + j];
    const R piv = *pp;
    const R w = fma(sc, tot, piv);
    *pp = fma(-tau, w, piv);
    cfv = tau * sc * w;
  }
  R cf[NA];
#pragma unroll
  for (int a = 0; a < NA; ++a) cf[a] = __shfl_sync(kFull, cfv, treduce32_lane<KP>(a));
  __syncwarp();
#define TSQR_WUPD(r)                                                                        \
  {                                                                                         \
    const int i = lo + lane + 32 * (r);                                                     \
    if (i < hi) {                                                                           \
      _Pragma("unroll") for (int a = 0; a < NA; ++a) Bc[a * ldt + i] = fma(-cf[a], xv[r], Bc[a * ldt + i]); \
    }                                                                                       \
  }
  TSQR_ROW_SLOTS(ra, RW, TSQR_WUPD)
#undef TSQR_WUPD
  __syncwarp();
}

// Lane l handles rows lo + l + 32 r of each reflector's tail (RW slots at most, entered
// through TSQR_ROW_SLOTS so only the needed slots issue); the K columns of B are exact.
template <int K, int RW, typename R>
__global__ void __launch_bounds__(128, 2) k_apply_warp(const ApplyParamsT<R> p, int njobs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  R *sm = reinterpret_cast<R *>(smraw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int jid = blockIdx.x * 4 + warp;
  if (jid >= njobs) return;  // warp-uniform; this kernel uses no block barrier
  const int n = p.n, ldt = p.ldt;
  R *Bt = sm + (size_t)warp * ((size_t)ldt + n) * K;  // tile rows, column-major
  R *PR = Bt + (size_t)ldt * K;                        // pivot rows, PR[c*n + j]
  TSQR_CHECK_OR_SKIP(p.njobs == 0 || p.job0 + jid < p.njobs, p.err)
  const JobDesc job = p.jobs[p.job0 + jid];
  const int64_t pr = job.piv_row;
  auto bcol = [&](int c) -> R * { return p.B + (int64_t)(p.col0 + c) * p.ldb; };
  TSQR_CHECK_OR_SKIP(pr >= 0 && (p.rows == 0 || pr + n <= p.rows) &&
                         (p.ntiles == 0 || job.tile_begin + job.tile_count <= p.ntiles),
                     p.err)

#pragma unroll
  for (int c = 0; c < K; ++c)
    for (int j = lane; j < n; j += 32) PR[c * n + j] = bcol(c)[pr + j];
  __syncwarp();

  const int nt = job.tile_count;
  for (int q = 0; q < nt; ++q) {
    const int tt = p.trans ? q : nt - 1 - q;
    const TileDesc td = p.tiles[job.tile_begin + tt];
    const int ht = td.nrows, kind = td.kind;
    const bool ge = (kind == GEQRT);
    const int64_t r0 = td.row0;
    TSQR_CHECK_OR_SKIP(r0 >= 0 && ht >= 1 && ht <= ldt && (p.rows == 0 || r0 + ht <= p.rows) && td.refl >= 0 &&
                           (p.nrefl == 0 || td.refl + n <= p.nrefl),
                       p.err)
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const R *src = bcol(c) + r0;
      for (int i = lane; i < ht; i += 32)
        Bt[c * ldt + i] = (ge && i < n) ? PR[c * n + i] : (p.formq ? R(0) : src[i]);
    }
    __syncwarp();

    const R *Vt = p.V + r0;
    // the next D reflectors' tails (and tau, scale) are in flight while one is applied:
    // each step is a short dependent chain, so one reflector ahead leaves HBM latency
    // exposed
    constexpr int D = RW <= 8 ? 4 : 2;
    R xb[D][RW], tb[D], sb[D];
    auto load_refl = [&](R(&dst)[RW], R &tau_d, R &scl_d, int s) {
      const int j = p.trans ? s : n - 1 - s;
      int lo, hi;
      refl_rows(kind, j, ht, lo, hi, td.off);
#pragma unroll
      for (int r = 0; r < RW; ++r) {
        const int i = lo + lane + 32 * r;
        dst[r] = (i < hi) ? __ldg(Vt + i + (int64_t)j * p.ldv) : R(0);
      }
      tau_d = __ldg(p.tau + td.refl + j);
      scl_d = __ldg(p.scl + td.refl + j);
    };
    // forming Q (reverse order), the reflectors j >= col0 + K change none of the pass's
    // columns: the pass starts after them
    const int s_beg = (p.formq && !p.trans) ? max(0, n - (p.col0 + K)) : 0;
#pragma unroll
    for (int d = 0; d < D; ++d)
      if (s_beg + d < n) load_refl(xb[d], tb[d], sb[d], s_beg + d);
    for (int s0 = s_beg; s0 < n; s0 += D) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int s = s0 + d;
        if (s >= n) break;
        const int j = p.trans ? s : n - 1 - s;
        int lo, hi;
        refl_rows(kind, j, ht, lo, hi, td.off);
        const R(&xv)[RW] = xb[d];
        const R tau = tb[d], sc = sb[d];
        // forming Q, reflector j leaves the pass's columns below j unchanged
        const int c0 = p.formq ? max(0, j - p.col0) : 0;
        switch (K - c0) {
          case 8: if (K >= 8) warp_reflector<(K >= 8 ? 8 : 1), RW, R>(Bt, PR, ldt, n, c0, ge, j, lo, hi, lane, xv, tau, sc); break;
          case 7: if (K >= 7) warp_reflector<(K >= 7 ? 7 : 1), RW, R>(Bt, PR, ldt, n, c0, ge, j, lo, hi, lane, xv, tau, sc); break;
          case 6: if (K >= 6) warp_reflector<(K >= 6 ? 6 : 1), RW, R>(Bt, PR, ldt, n, c0, ge, j, lo, hi, lane, xv, tau, sc); break;
          case 5: if (K >= 5) warp_reflector<(K >= 5 ? 5 : 1), RW, R>(Bt, PR, ldt, n, c0, ge, j, lo, hi, lane, xv, tau, sc); break;
          case 4: if (K >= 4) warp_reflector<(K >= 4 ? 4 : 1), RW, R>(Bt, PR, ldt, n, c0, ge, j, lo, hi, lane, xv, tau, sc); break;
          case 3: if (K >= 3) warp_reflector<(K >= 3 ? 3 : 1), RW, R>(Bt, PR, ldt, n, c0, ge, j, lo, hi, lane, xv, tau, sc); break;
          case 2: if (K >= 2) warp_reflector<(K >= 2 ? 2 : 1), RW, R>(Bt, PR, ldt, n, c0, ge, j, lo, hi, lane, xv, tau, sc); break;
          case 1: warp_reflector<1, RW, R>(Bt, PR, ldt, n, c0, ge, j, lo, hi, lane, xv, tau, sc); break;
          default: break;
        }
        if (s + D < n) load_refl(xb[d], tb[d], sb[d], s + D);
      }
    }
#pragma unroll
    for (int c = 0; c < K; ++c) {
      R *dst = bcol(c) + r0;
      for (int i = lane; i < ht; i += 32) {
        if (ge && i < n)
          PR[c * n + i] = Bt[c * ldt + i];
        else
          dst[i] = Bt[c * ldt + i];
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int c = 0; c < K; ++c)
    for (int j = lane; j < n; j += 32) bcol(c)[pr + j] = PR[c * n + j];
}

// ------------------------------------------- one column: tile pairs per warp
// Q^T b or Q b for a single column is, per reflector, a dot product over the tile rows, a
// reduction and an update of one vector. With a whole warp on one tile (k_apply_warp) a
// lane holds about five rows of a 144-row tile, and the FP64 pipe spends as much on the
// 32-lane reduction and the scalar step as on the dot product and the update. Here a job's
// tiles are dealt alternately to the two half-warps: half 1 runs the next tile in the
// processing order one reflector step behind half 0. Reflector j of a tile needs only the
// pivot entry PR[j] as the previous tile's reflector j left it (and reflectors j' > j do
// not touch it), so the lag of one step is enough. Each warp instruction then carries two
// reflector applications, each lane holds about ten rows, and a reduction spans 16 lanes.
//
// Half h runs local steps u = 0, 1, ...: tile position q = 2 (u / n) + h, reflector step
// u mod n, at warp step t = u + h. The pivot entries live in two buffers: tile q reads
// buffer q mod 2 and writes the other, so no entry is rewritten in the step that reads it,
// and the final pivot rows are in buffer nt mod 2. A leaf tile (GEQRT) holds the pivot
// rows themselves: applying Q^T (the leaf first) it starts from the input buffer and
// publishes row j after reflector j (later reflectors touch rows > j only); applying Q
// (the leaf last) it takes row j from the input buffer at reflector j (reflectors j' > j,
// which run before, touch rows >= j' only) and writes its rows < n out at the end.

template <int RV>
__global__ void __launch_bounds__(128, 3) k_apply_vec(const ApplyParamsT<double> p, int njobs) {
  // reflector tails loaded ahead per half (fewer for tall tiles, to stay in registers)
  constexpr int kVecD = RV <= 16 ? 3 : 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int h = lane >> 4, hl = lane & 15;
  const int jid = blockIdx.x * 4 + warp;
  if (jid >= njobs) return;  // warp-uniform; this kernel uses no block barrier
  const int n = p.n, ldt = p.ldt;
  double *PR = reinterpret_cast<double *>(smraw) + (size_t)warp * (2 * (size_t)ldt + 2 * n);  // 2 x n
  double *Bt = PR + 2 * n + (size_t)h * ldt;  // this half's tile
  double *B = p.B + (int64_t)p.col0 * p.ldb;
  TSQR_CHECK_OR_SKIP(p.njobs == 0 || p.job0 + jid < p.njobs, p.err)
  const JobDesc job = p.jobs[p.job0 + jid];
  const int64_t pr = job.piv_row;
  const int nt = job.tile_count;
  TSQR_CHECK_OR_SKIP(pr >= 0 && (p.rows == 0 || pr + n <= p.rows) &&
                         (p.ntiles == 0 || job.tile_begin + nt <= p.ntiles),
                     p.err)
#ifdef TSQR_CHECK
  // every tile is checked before the pipeline starts: a check inside it would let one half
  // leave while the other waits for it in a shuffle
  for (int q = 0; q < nt; ++q) {
    const TileDesc tq = p.tiles[job.tile_begin + q];
    TSQR_CHECK_OR_SKIP(tq.row0 >= 0 && tq.nrows >= 1 && tq.nrows <= ldt &&
                           (p.rows == 0 || tq.row0 + tq.nrows <= p.rows) && tq.refl >= 0 &&
                           (p.nrefl == 0 || tq.refl + n <= p.nrefl),
                       p.err)
  }
#endif
  for (int j = lane; j < n; j += 32) PR[j] = B[pr + j];

  const int usteps = ((nt - h + 1) >> 1) * n;                 // this half's local steps
  const int T = max(((nt + 1) >> 1) * n, (nt >> 1) * n + 1);  // warp steps
  auto tile_of = [&](int u) -> TileDesc {
    const int q = 2 * (u / n) + h;
    return p.tiles[job.tile_begin + (p.trans ? q : nt - 1 - q)];
  };
  auto refl_of = [&](int u) -> int { return p.trans ? u % n : n - 1 - u % n; };
  // this lane's rows of the tail of local step u's reflector, its tau, scale, tau * scale
  double xb[kVecD][RV], tb[kVecD], sb[kVecD], cb[kVecD];
  auto load = [&](int d, int u) {
#pragma unroll
    for (int r = 0; r < RV; ++r) xb[d][r] = 0.0;
    tb[d] = sb[d] = cb[d] = 0.0;
    if (u < 0 || u >= usteps) return;
    const TileDesc tq = tile_of(u);
    const int j = refl_of(u);
    int lo, hi;
    refl_rows(tq.kind, j, tq.nrows, lo, hi, tq.off);
    const double *v = p.V + tq.row0 + (int64_t)j * p.ldv;
#pragma unroll
    for (int r = 0; r < RV; ++r) {
      const int i = lo + hl + 16 * r;
      if (i < hi) xb[d][r] = __ldg(v + i);
    }
    tb[d] = __ldg(p.tau + tq.refl + j);
    sb[d] = __ldg(p.scl + tq.refl + j);
    cb[d] = tb[d] * sb[d];
  };
#pragma unroll
  for (int d = 0; d < kVecD; ++d) load(d, d - h);

  TileDesc td{};  // the half's current tile
  double *Pin = PR, *Pout = PR + n;  // its pivot buffers (tile q: in = q mod 2)
  // A tile leaves shared memory at the warp step after its last reflector (the rows of
  // that update belong to other lanes); the leaf's pivot rows go back to PR (applying Q)
  // or were published row by row (applying Q^T).
  auto store_prev = [&](int u) {
    const int up = u - 1;
    if (up < 0 || up >= usteps || up % n != n - 1) return;
    const bool ge = (td.kind == GEQRT);
    for (int i = hl; i < td.nrows; i += 16) {
      if (ge && i < n) {
        if (!p.trans) Pout[i] = Bt[i];
      } else {
        B[td.row0 + i] = Bt[i];
      }
    }
  };
  for (int t0 = 0; t0 < T; t0 += kVecD) {
#pragma unroll
    for (int d = 0; d < kVecD; ++d) {
      const int t = t0 + d;
      if (t >= T) break;  // warp-uniform
      const int u = t - h;
      const bool act = (u >= 0 && u < usteps);
      __syncwarp();  // the previous step's updates and head entries are visible
      store_prev(u);
      if (act && u % n == 0) {  // stage the next tile
        td = tile_of(u);
        const int q = 2 * (u / n) + h;
        Pin = PR + (q & 1) * n;
        Pout = PR + ((q + 1) & 1) * n;
        const bool ge = (td.kind == GEQRT);
        for (int i = hl; i < td.nrows; i += 16) {
          if (ge && i < n) {
            if (p.trans) Bt[i] = Pin[i];
          } else {
            Bt[i] = B[td.row0 + i];
          }
        }
      }
      __syncwarp();
      const int j = refl_of(act ? u : 0);
      int lo = 0, hi = 0;
      if (act) refl_rows(td.kind, j, td.nrows, lo, hi, td.off);
      const int rh = (hi - lo + 15) >> 4;
      const int ra = max(rh, __shfl_xor_sync(kFull, rh, 16));
      const double(&xv)[RV] = xb[d];
      double acc = 0.0;
#define TSQR_VDOT(r)                                                                         \
  {                                                                                          \
    const int i = lo + hl + 16 * (r);                                                        \
    if (i < hi) acc = fma(xv[r], Bt[i], acc);                                                \
  }
      TSQR_ROW_SLOTS(ra, RV, TSQR_VDOT)
#undef TSQR_VDOT
#pragma unroll
      for (int m = 8; m >= 1; m >>= 1) acc += __shfl_xor_sync(kFull, acc, m);
      if (act) {
        // v = [1; scale * tail]: w = v^T b, the head entry becomes piv - tau w and the tail
        // rows take b_i - (tau scale w) x_i
        const bool ge = (td.kind == GEQRT);
        const double piv = (ge && p.trans) ? Bt[j] : Pin[j];
        const double w = fma(sb[d], acc, piv);
        const double cf = cb[d] * w;
#define TSQR_VUPD(r)                                                                         \
  {                                                                                          \
    const int i = lo + hl + 16 * (r);                                                        \
    if (i < hi) Bt[i] = fma(-cf, xv[r], Bt[i]);                                              \
  }
        TSQR_ROW_SLOTS(ra, RV, TSQR_VUPD)
#undef TSQR_VUPD
        if (hl == 0) {
          const double np = fma(-tb[d], w, piv);
          if (ge && !p.trans)
            Bt[j] = np;  // later reflectors j' < j update row j as a tail row
          else
            Pout[j] = np;
        }
      }
      load(d, u + kVecD);
    }
  }
  __syncwarp();
  store_prev(T - h);
  __syncwarp();
  const double *Pf = PR + (nt & 1) * n;
  for (int j = lane; j < n; j += 32) B[pr + j] = Pf[j];
}

// ------------------------------------------------------------ one CTA per job
// The structure of the factor kernel: the job's tile of B (up to 16*CMAX columns of this
// pass) is staged in shared memory, the pivot row of each reflector is staged from
// global memory (prefetched one reflector ahead), and the reflector tail is prefetched
// into registers (every half-warp reads the same rows, so the loads hit L1). The
// half-warp of rank h owns columns cs + h + 16 t; each warp issues exactly its own slots.
// The ranks rotate with the reflector (warp w has rank (w + s) mod 8 at reflector step s):
// a CTA's warp w always runs on SM sub-partition w mod 4, and with a fixed order the
// lowest warps, which take the extra slots of uneven steps, would load the same
// sub-partition's FP64 pipe in every CTA on the SM. Warp 0 runs each step's scalar phase.
constexpr int kTileThreads = 256;


__device__ __forceinline__ int warp_slots(int cs, int nc, int warp) {
  const int r = nc - cs - 2 * warp;
  return r <= 0 ? 0 : (r + 15) >> 4;
}

// dots: PC[c] = sum_r xv[r] * Bt[c][lo + hl + 16 r] over rows < hi, c = cs + hw + 16 t
template <int NS, int RM, typename R>
__device__ __forceinline__ void tile_dots(const R *__restrict__ Bt, int ldt, int cs, int kc, int lo,
                                          int hi, int hw, int hl, const R (&xv)[RM],
                                          R *__restrict__ PC) {
  constexpr int C = pow2ceil(NS);
  const int cb = cs + hw;
  R acc[C];
#pragma unroll
  for (int t = 0; t < C; ++t) acc[t] = R(0);
  const int ra = (hi - lo + 15) >> 4;
#define TSQR_DOT_ROW(r)                                                                    \
  {                                                                                          \
    const int i = lo + hl + 16 * (r);                                                        \
    if (i < hi) {                                                                            \
      _Pragma("unroll") for (int t = 0; t < NS; ++t) {                                       \
        const int c = cb + 16 * t;                                                           \
        if (t < NS - 1 || c < kc) acc[t] = fma(xv[r], Bt[(size_t)c * ldt + i], acc[t]);     \
      }                                                                                      \
    }                                                                                        \
  }
  TSQR_ROW_SLOTS(ra, RM, TSQR_DOT_ROW)
#undef TSQR_DOT_ROW
  int idx;
  const R sres = treduce16<C, R>(acc, hl, idx);
  const int c = cb + 16 * idx;
  if ((hl & (16 / C - 1)) == 0 && idx < NS && c < kc) PC[c] = sres;
}

template <int NS, int RM, typename R>
__device__ __forceinline__ void tile_update(R *__restrict__ Bt, int ldt, int cs, int kc, int lo, int hi,
                                           int hw, int hl, const R (&xv)[RM],
                                           const R *__restrict__ CF) {
  const int cb = cs + hw;
  R cf[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    const int c = cb + 16 * t;
    cf[t] = (c < kc) ? CF[c] : R(0);
  }
  const int ra = (hi - lo + 15) >> 4;
#define TSQR_UPD_ROW(r)                                                                    \
  {                                                                                          \
    const int i = lo + hl + 16 * (r);                                                        \
    if (i < hi) {                                                                            \
      _Pragma("unroll") for (int t = 0; t < NS; ++t) {                                       \
        const int c = cb + 16 * t;                                                           \
        if (t < NS - 1 || c < kc) {                                                          \
          R *b = Bt + (size_t)c * ldt + i;                                                   \
          *b = fma(-cf[t], xv[r], *b);                                                       \
        }                                                                                    \
      }                                                                                      \
    }                                                                                        \
  }
  TSQR_ROW_SLOTS(ra, RM, TSQR_UPD_ROW)
#undef TSQR_UPD_ROW
}

template <int CMAX, int RM, typename R>
__device__ __forceinline__ void dots_dispatch(const R *Bt, int ldt, int cs, int kc, int lo, int hi, int hw,
                                              int hl, int warp, const R (&xv)[RM], R *PC) {
  switch (warp_slots(cs, kc, warp)) {
    case 0: return;
    case 1: tile_dots<1, RM, R>(Bt, ldt, cs, kc, lo, hi, hw, hl, xv, PC); return;
    case 2: if (CMAX >= 2) tile_dots<(CMAX >= 2 ? 2 : 1), RM>(Bt, ldt, cs, kc, lo, hi, hw, hl, xv, PC); return;
    case 3: if (CMAX >= 4) tile_dots<(CMAX >= 4 ? 3 : 1), RM>(Bt, ldt, cs, kc, lo, hi, hw, hl, xv, PC); return;
    default: if (CMAX >= 4) tile_dots<(CMAX >= 4 ? 4 : 1), RM>(Bt, ldt, cs, kc, lo, hi, hw, hl, xv, PC); return;
  }
}

template <int CMAX, int RM, typename R>
__device__ __forceinline__ void update_dispatch(R *Bt, int ldt, int cs, int kc, int lo, int hi, int hw,
                                                int hl, int warp, const R (&xv)[RM], const R *CF) {
  switch (warp_slots(cs, kc, warp)) {
    case 0: return;
    case 1: tile_update<1, RM, R>(Bt, ldt, cs, kc, lo, hi, hw, hl, xv, CF); return;
    case 2: if (CMAX >= 2) tile_update<(CMAX >= 2 ? 2 : 1), RM>(Bt, ldt, cs, kc, lo, hi, hw, hl, xv, CF); return;
    case 3: if (CMAX >= 4) tile_update<(CMAX >= 4 ? 3 : 1), RM>(Bt, ldt, cs, kc, lo, hi, hw, hl, xv, CF); return;
    default: if (CMAX >= 4) tile_update<(CMAX >= 4 ? 4 : 1), RM>(Bt, ldt, cs, kc, lo, hi, hw, hl, xv, CF); return;
  }
}

// MINB: CTAs per SM the launch is planned for (3 only with 144-row tiles, RM = 9).
template <int CMAX, int RM, typename R, int MINB>
__global__ void __launch_bounds__(kTileThreads, MINB) k_apply_tile(const ApplyParamsT<R> p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  R *sm = reinterpret_cast<R *>(smraw);
  constexpr int KC = 16 * CMAX;
  const int n = p.n, ldt = p.ldt;
  const int col0 = p.col0 + blockIdx.y * KC;
  const int kc = min(KC, p.k - (int)blockIdx.y * KC);
  R *Bt = sm;                        // KC columns of ldt rows
  R *PC = Bt + (size_t)KC * ldt;     // dot products, then update coefficients
  R *PV = PC + KC;                   // staged pivot row (TSQRT / TTQRT)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int hw = tid >> 4, hl = tid & 15;
  TSQR_CHECK_OR_SKIP(p.njobs == 0 || p.job0 + (int)blockIdx.x < p.njobs, p.err)
  const JobDesc job = p.jobs[p.job0 + blockIdx.x];
  const int64_t pr = job.piv_row;
  auto bp = [&](int64_t row, int c) -> R * { return p.B + row + (int64_t)(col0 + c) * p.ldb; };
  constexpr int PFN = (KC + 31) / 32;
  TSQR_CHECK_OR_SKIP(pr >= 0 && (p.rows == 0 || pr + n <= p.rows) &&
                         (p.ntiles == 0 || job.tile_begin + job.tile_count <= p.ntiles),
                     p.err)

  const int nt = job.tile_count;
  for (int q = 0; q < nt; ++q) {
    const int tt = p.trans ? q : nt - 1 - q;
    const TileDesc td = p.tiles[job.tile_begin + tt];
    const int ht = td.nrows, kind = td.kind;
    const bool ge = (kind == GEQRT);
    const int64_t r0 = td.row0;
    TSQR_CHECK_OR_SKIP(r0 >= 0 && ht >= 1 && ht <= ldt && (p.rows == 0 || r0 + ht <= p.rows) && td.refl >= 0 &&
                           (p.nrefl == 0 || td.refl + n <= p.nrefl),
                       p.err)
    const R *Vt = p.V + r0;
    // stage the tile: when forming Q every row below the pivot block starts at zero
    for (int c = warp; c < kc; c += kTileThreads / 32) {
      const R *src = bp(r0, c);
      R *dst = Bt + (size_t)c * ldt;
      for (int i = lane; i < ht; i += 32) dst[i] = (p.formq && !(ge && i < n)) ? R(0) : src[i];
    }
    const int j0 = p.trans ? 0 : n - 1;
    if (!ge)
      for (int c = tid; c < kc; c += kTileThreads) PV[c] = __ldcg(bp(pr + j0, c));
    R xv[RM], xn[RM];
    // warp 0 holds the current reflector's scalars and loads the next one's a step ahead
    R tau = R(0), sc = R(0), tau_n = R(0), sc_n = R(0);
    if (warp == 0) {
      tau = __ldg(p.tau + td.refl + j0);
      sc = __ldg(p.scl + td.refl + j0);
    }
    {
      int lo, hi;
      refl_rows(kind, j0, ht, lo, hi, td.off);
#pragma unroll
      for (int r = 0; r < RM; ++r) {
        const int i = lo + hl + 16 * r;
        xv[r] = (i < hi) ? __ldg(Vt + i + (int64_t)j0 * p.ldv) : R(0);
      }
    }
    __syncthreads();

    for (int s = 0; s < n; ++s) {
      const int j = p.trans ? s : n - 1 - s;
      const bool more = (s + 1 < n);
      const int jn = p.trans ? s + 1 : n - 2 - s;
      int lo, hi;
      refl_rows(kind, j, ht, lo, hi, td.off);
      const int cs = p.formq ? max(0, j - col0) : 0;  // first column this reflector touches
      // prefetch the next reflector's tail (registers) and pivot row (warp 1)
      if (more) {
        if (warp == 0) {
          tau_n = __ldg(p.tau + td.refl + jn);
          sc_n = __ldg(p.scl + td.refl + jn);
        }
        int lo2, hi2;
        refl_rows(kind, jn, ht, lo2, hi2, td.off);
#pragma unroll
        for (int r = 0; r < RM; ++r) {
          const int i = lo2 + hl + 16 * r;
          xn[r] = (i < hi2) ? __ldg(Vt + i + (int64_t)jn * p.ldv) : R(0);
        }
      }
      R pf[PFN];
      const bool do_pf = (!ge) && warp == 1 && more;
      if (do_pf) {
#pragma unroll
        for (int u = 0; u < PFN; ++u) {
          const int c = lane + 32 * u;
          pf[u] = (c < kc) ? __ldcg(bp(pr + jn, c)) : R(0);
        }
      }
      // this reflector's rank of the warp; warp 0 keeps the scalar phase
      const int rw = (warp + s) & 7;
      const int hr = 2 * rw + (hw & 1);
      if (cs < kc) {
        dots_dispatch<CMAX, RM, R>(Bt, ldt, cs, kc, lo, hi, hr, hl, rw, xv, PC);
        __syncthreads();
        if (warp == 0) {
          const R ts = tau * sc;
          for (int c = cs + lane; c < kc; c += 32) {
            const R piv = ge ? Bt[(size_t)c * ldt + j] : PV[c];
            const R w = fma(sc, PC[c], piv);
            const R np = fma(-tau, w, piv);
            PC[c] = ts * w;
            if (ge)
              Bt[(size_t)c * ldt + j] = np;
            else
              *bp(pr + j, c) = np;
          }
        }
        __syncthreads();
        update_dispatch<CMAX, RM, R>(Bt, ldt, cs, kc, lo, hi, hr, hl, rw, xv, PC);
      }
      if (do_pf) {
#pragma unroll
        for (int u = 0; u < PFN; ++u) {
          const int c = lane + 32 * u;
          if (c < kc) PV[c] = pf[u];
        }
      }
#pragma unroll
      for (int r = 0; r < RM; ++r) xv[r] = xn[r];
      tau = tau_n;
      sc = sc_n;
      __syncthreads();
    }
    for (int c = warp; c < kc; c += kTileThreads / 32) {
      R *dst = bp(r0, c);
      const R *src = Bt + (size_t)c * ldt;
      for (int i = lane; i < ht; i += 32) dst[i] = src[i];
    }
    __syncthreads();
  }
}

// ------------------------------------------ cluster tier: pipelined tree levels of Q B
// B <- Q B (and the thin Q) through three binary tree levels in one launch of clusters of
// kClusterSize CTAs, the mirror of the factorization's cluster tier: the levels run top
// down, and a node applies its reflectors n-1 .. 0 to [pivot block; tile block] of 16
// columns. Reflector j touches pivot row j and tile rows 0..j, so after the node's step s
// (reflector n-1-s) row n-1-s of both blocks is final; a child's step s needs exactly that
// row of its parent's block (its pivot rows are the parent's pivot rows or tile rows). The
// copy warp of the child waits for the parent's progress counter and copies the row for the
// next step from the parent's shared memory (distributed shared memory) while the other
// warps run the current step. Each block goes to global memory once, from the CTA that
// finishes it (a block whose rows an in-cluster child takes over is left to that child).
constexpr int kClusterCols = 16;
constexpr int kApplyClusterThreads = kTileThreads + 32;

template <int RM>
__device__ __forceinline__ void apply_node_cluster(const ApplyParamsT<double> &p, const JobDesc job,
                                                   const ApplyClusterSlot sl, unsigned char *smraw, unsigned *done,
                                                   int *gave_up) {
  using R = double;
  constexpr int KC = kClusterCols, KCP = KC + 1;
  R *sm = reinterpret_cast<R *>(smraw);
  const int n = p.n, ldt = n;
  const int col0 = p.col0 + blockIdx.y * KC;
  const int kc = min(KC, p.k - (int)blockIdx.y * KC);
  R *Bt = sm;                     // the tile block: KC columns of n rows
  R *PC = Bt + (size_t)KC * ldt;  // dot products, then update coefficients
  R *P = PC + KC;                 // the pivot block, row-major: P[i * KCP + c]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int hw = tid >> 4, hl = tid & 15;
  const bool cw = (warp == kTileThreads / 32);
  const TileDesc td = p.tiles[job.tile_begin];
  const int64_t pr = job.piv_row, r0 = td.row0;
  TSQR_CHECK_OR_SKIP(job.tile_count == 1 && td.kind == TTQRT && td.nrows == n && td.off == 0 && pr >= 0 &&
                         r0 >= 0 && (p.rows == 0 || (pr + n <= p.rows && r0 + n <= p.rows)) && td.refl >= 0 &&
                         (p.nrefl == 0 || td.refl + n <= p.nrefl) && sl.parent >= -1 &&
                         sl.parent < kClusterSize && kc >= 1,
                     p.err)
  auto bp = [&](int64_t row, int c) -> R * { return p.B + row + (int64_t)(col0 + c) * p.ldb; };
  const uint32_t a_done = smem_u32(done), a_P = smem_u32(P), a_T = smem_u32(Bt);
  // the copy warp: row `row` of the parent's block, final once the parent has finished its
  // step n - 1 - row
  auto fetch_row = [&](int row) {
    if (!*gave_up) {
      const uint32_t a = cluster_map(a_done, sl.parent);
      uint32_t it = 0;
      while (ld_acquire_cluster_u32(a) < (uint32_t)(n - row)) {
        if (++it > kClusterSpinLimit) {
          if (lane == 0) atomicOr(p.err, kErrTimeout);
          *gave_up = 1;
          break;
        }
        __nanosleep(32);
      }
    }
    __syncwarp();
    for (int c = lane; c < kc; c += 32) {
      const uint32_t src = sl.side == 0 ? a_P + (uint32_t)(sizeof(R) * (row * KCP + c))
                                        : a_T + (uint32_t)(sizeof(R) * ((size_t)c * ldt + row));
      P[row * KCP + c] = ld_cluster_f64(cluster_map(src, sl.parent));
    }
  };

  // the tile block starts at B's rows (zero when forming Q); the pivot block is complete in
  // global memory when the parent ran in an earlier launch, else it arrives row by row
  for (int c = warp; c < kc; c += kApplyClusterThreads / 32)
    for (int i = lane; i < n; i += 32) Bt[(size_t)c * ldt + i] = p.formq ? R(0) : *bp(r0 + i, c);
  if (sl.parent < 0) {
    for (int e = tid; e < n * kc; e += kApplyClusterThreads) {
      const int i = e % n, c = e / n;
      P[i * KCP + c] = __ldcg(bp(pr + i, c));
    }
  } else if (cw) {
    fetch_row(n - 1);
  }
  const R *Vt = p.V + r0;
  R xv[RM], xn[RM];
  R tau = R(0), sc = R(0), tau_n = R(0), sc_n = R(0);
  if (warp == 0) {
    tau = __ldg(p.tau + td.refl + n - 1);
    sc = __ldg(p.scl + td.refl + n - 1);
  }
#pragma unroll
  for (int r = 0; r < RM; ++r) {
    const int i = hl + 16 * r;
    xv[r] = (!cw && i < n) ? __ldg(Vt + i + (int64_t)(n - 1) * p.ldv) : R(0);
  }
  __syncthreads();

  for (int s = 0; s < n; ++s) {
    const int j = n - 1 - s, jn = j - 1;
    const bool more = (s + 1 < n);
    const int lo = 0, hi = j + 1;  // reflector j's tail: tile rows 0..j
    const int cs = p.formq ? max(0, j - col0) : 0;
    if (cw) {
      if (more && sl.parent >= 0) fetch_row(jn);
    } else if (more) {
      if (warp == 0) {
        tau_n = __ldg(p.tau + td.refl + jn);
        sc_n = __ldg(p.scl + td.refl + jn);
      }
#pragma unroll
      for (int r = 0; r < RM; ++r) {
        const int i = hl + 16 * r;
        xn[r] = (i <= jn) ? __ldg(Vt + i + (int64_t)jn * p.ldv) : R(0);
      }
    }
    const int rw = (warp + s) & 7;
    const int hr = 2 * rw + (hw & 1);
    if (cs < kc) {
      if (!cw) dots_dispatch<1, RM, R>(Bt, ldt, cs, kc, lo, hi, hr, hl, rw, xv, PC);
      __syncthreads();
      if (warp == 0) {
        const R ts = tau * sc;
        for (int c = cs + lane; c < kc; c += 32) {
          const R piv = P[j * KCP + c];
          const R w = fma(sc, PC[c], piv);
          PC[c] = ts * w;
          P[j * KCP + c] = fma(-tau, w, piv);
        }
      }
      __syncthreads();
      if (!cw) update_dispatch<1, RM, R>(Bt, ldt, cs, kc, lo, hi, hr, hl, rw, xv, PC);
    }
    if (!cw) {
#pragma unroll
      for (int r = 0; r < RM; ++r) xv[r] = xn[r];
      tau = tau_n;
      sc = sc_n;
    }
    __syncthreads();
    if (tid == 0) st_release_cluster_u32(a_done, (uint32_t)(s + 1));
  }
  // each block to global memory unless an in-cluster child takes its rows over
  if (!(sl.kids & 1))
    for (int e = tid; e < n * kc; e += kApplyClusterThreads) {
      const int i = e % n, c = e / n;
      *bp(pr + i, c) = P[i * KCP + c];
    }
  if (!(sl.kids & 2))
    for (int c = warp; c < kc; c += kApplyClusterThreads / 32)
      for (int i = lane; i < n; i += 32) *bp(r0 + i, c) = Bt[(size_t)c * ldt + i];
}

template <int RM>
__global__ void __launch_bounds__(kApplyClusterThreads, 2)
    k_apply_cluster(const ApplyParamsT<double> p, const ApplyClusterSlot *__restrict__ slots) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ unsigned s_done;
  __shared__ int s_gave_up;
  const ApplyClusterSlot sl = slots[blockIdx.x];
  if (threadIdx.x == 0) {
    s_done = 0;
    s_gave_up = 0;
  }
  cluster_barrier();  // every counter is initialised before any child polls it
  if (sl.job >= 0) apply_node_cluster<RM>(p, p.jobs[sl.job], sl, smraw, &s_done, &s_gave_up);
  cluster_barrier();  // no CTA leaves while a child may still read its shared memory
}

template <int CMAX, int RM, typename R, int MINB>
cudaError_t launch_tile_t(const ApplyParamsT<R> &p, int njobs, cudaStream_t s) {
  constexpr int KC = 16 * CMAX;
  const size_t bytes = sizeof(R) * ((size_t)KC * p.ldt + 2 * KC);
  cudaError_t e = cudaFuncSetAttribute(k_apply_tile<CMAX, RM, R, MINB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  dim3 grid(njobs, (p.k + KC - 1) / KC);
  k_apply_tile<CMAX, RM, R, MINB><<<grid, kTileThreads, bytes, s>>>(p);
  return cudaGetLastError();
}

// Rows per lane (RM) sized to the tile; the three-CTA build exists for 144-row tiles.
template <int CMAX, typename R>
cudaError_t launch_tile_rm(const ApplyParamsT<R> &p, int njobs, int ctas_per_sm, cudaStream_t s) {
  const int rows_per_lane = (p.ldt + 15) / 16;
  if (rows_per_lane <= 8) return launch_tile_t<CMAX, 8, R, 2>(p, njobs, s);
  if (rows_per_lane <= 9)
    return ctas_per_sm >= 3 ? launch_tile_t<CMAX, 9, R, 3>(p, njobs, s) : launch_tile_t<CMAX, 9, R, 2>(p, njobs, s);
  if (rows_per_lane <= 16) return launch_tile_t<CMAX, 16, R, 2>(p, njobs, s);
  return launch_tile_t<CMAX, 32, R, 1>(p, njobs, s);
}

template <int K, int RW, typename R>
cudaError_t launch_warp_t(const ApplyParamsT<R> &p, int njobs, cudaStream_t s) {
  const size_t bytes = sizeof(R) * 4 * ((size_t)p.ldt + p.n) * K;
  cudaError_t e = cudaFuncSetAttribute(k_apply_warp<K, RW, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return e;
  k_apply_warp<K, RW, R><<<(njobs + 3) / 4, 128, bytes, s>>>(p, njobs);
  return cudaGetLastError();
}

template <int K, typename R>
cudaError_t launch_warp_k(const ApplyParamsT<R> &p, int njobs, cudaStream_t s) {
  if (p.ldt <= 256) return launch_warp_t<K, 8, R>(p, njobs, s);
  return launch_warp_t<K, 16, R>(p, njobs, s);
}

template <int RV>
cudaError_t launch_vec_t(const ApplyParamsT<double> &p, int njobs, cudaStream_t s) {
  const size_t bytes = sizeof(double) * 4 * (2 * (size_t)p.ldt + 2 * (size_t)p.n);
  cudaError_t e = cudaFuncSetAttribute(k_apply_vec<RV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k_apply_vec<RV><<<(njobs + 3) / 4, 128, bytes, s>>>(p, njobs);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_apply_any(const ApplyParamsT<R> &p, int njobs, int ctas_per_sm, int cols_per_cta,
                             cudaStream_t s) {
  if (njobs <= 0 || p.k <= 0) return cudaSuccess;
  if (p.ldt > 512) return cudaErrorInvalidValue;
  if (p.k <= 8) {
    switch (p.k) {
      case 1: return launch_warp_k<1, R>(p, njobs, s);
      case 2: return launch_warp_k<2, R>(p, njobs, s);
      case 3: return launch_warp_k<3, R>(p, njobs, s);
      case 4: return launch_warp_k<4, R>(p, njobs, s);
      case 5: return launch_warp_k<5, R>(p, njobs, s);
      case 6: return launch_warp_k<6, R>(p, njobs, s);
      case 7: return launch_warp_k<7, R>(p, njobs, s);
      default: return launch_warp_k<8, R>(p, njobs, s);
    }
  }
  // up to 64 columns per CTA; fewer columns (or a cap) use a narrower tile and more CTAs
  if (p.k <= 16 || cols_per_cta <= 16) return launch_tile_rm<1, R>(p, njobs, ctas_per_sm, s);
  if (p.k <= 32 || cols_per_cta <= 32) return launch_tile_rm<2, R>(p, njobs, ctas_per_sm, s);
  return launch_tile_rm<4, R>(p, njobs, ctas_per_sm, s);
}

template <int RM>
cudaError_t launch_cluster_rm(const ApplyParamsT<double> &p, const ApplyClusterSlot *slots, int nclusters,
                              cudaStream_t s) {
  const size_t bytes = apply_cluster_smem_bytes(p.n);
  cudaError_t e = cudaFuncSetAttribute(k_apply_cluster<RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nclusters * kClusterSize), (unsigned)((p.k + kClusterCols - 1) / kClusterCols));
  cfg.blockDim = dim3(kApplyClusterThreads);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kClusterSize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_apply_cluster<RM>, p, slots);
}

}  // namespace

size_t apply_cluster_smem_bytes(int n) {
  return sizeof(double) * ((size_t)kClusterCols * n + kClusterCols + (size_t)n * (kClusterCols + 1));
}

cudaError_t launch_apply_cluster(const ApplyParamsT<double> &p, const ApplyClusterSlot *slots, int nclusters,
                                 cudaStream_t s) {
  if (nclusters <= 0 || p.k <= 0) return cudaSuccess;
  if (p.n <= 128) return launch_cluster_rm<8>(p, slots, nclusters, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_apply(const ApplyParamsT<double> &p, int njobs, cudaStream_t s, int ctas_per_sm,
                         int cols_per_cta, bool tile_pairs) {
  // one column of B over jobs of several tiles: the tile-pair kernel (its one-step lag
  // needs n >= 2; forming Q keeps the warp kernel)
  if (tile_pairs && p.k == 1 && !p.formq && p.n >= 2 && njobs > 0) {
    const int rows_per_lane = (p.ldt + 15) / 16;
    if (rows_per_lane <= 8) return launch_vec_t<8>(p, njobs, s);
    if (rows_per_lane <= 9) return launch_vec_t<9>(p, njobs, s);
    if (rows_per_lane <= 16) return launch_vec_t<16>(p, njobs, s);
    if (rows_per_lane <= 32) return launch_vec_t<32>(p, njobs, s);
    return cudaErrorInvalidValue;
  }
  return launch_apply_any(p, njobs, ctas_per_sm, cols_per_cta, s);
}

}  // namespace tsqr
