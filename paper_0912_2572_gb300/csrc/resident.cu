// The resident persistent kernel of the resident server (sm_103a; the paper has no
// counterpart). It runs the batched engine's jobs (k_factor_batch: FP64 and FP32 chains,
// the wait-free reduction tree, R and X of each request) and the refinement tasks of the
// mixed path (k_refine_batch) from three work rings: two the host appends requests' chain
// jobs to while the kernel runs (short requests, long ones) and one for the refinement
// tasks the kernel queues itself. The ring protocol is described with ResCtl in
// tsqr_internal.h.
//
// Every request's tables, counters and inputs live at addresses the host reuses for later
// requests while this kernel runs, so every such read goes through L2 (the COH builds of
// the job functions); an L1 line another request left behind is never read.
//
// Waits are bounded. A CTA that has claimed a device-ring entry waits for its producer to
// release it (a handful of stores away) at most kSeqWaitPolls polls, then sets the timeout
// bit of the device error word and drops the entry; the host then fails the requests in
// flight. A CTA that finds nothing to claim sleeps between polls (2-32 us); after
// idle_polls empty polls in a row, if no CTA is busy and every ring is empty, it ends
// the launch (quit); a CTA that has waited kIdleGiveUp polls ends it as well, whatever
// the others are doing, so no launch outlives a stalled request by much. Ending a launch
// loses nothing: entries not yet claimed stay in the rings for the next launch.
#include <cstdint>

#include "factor_job.cuh"
#include "refine_task.cuh"
#include "tsqr_internal.h"

namespace tsqr {
namespace {

constexpr int kResCmax = 16;            // column slots for up to 144 columns (n + k)
constexpr int64_t kSeqWaitPolls = 1 << 22;
constexpr int64_t kIdleGiveUp = 1 << 18;  // ~2-8 s of empty polls

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_i32(const int32_t *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_sys_i32(int32_t *p, int v) {
  asm volatile("st.release.sys.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// A struct of 8-byte words read through L2.
template <typename T>
__device__ __forceinline__ T ldcg_struct(const T *p) {
  static_assert(sizeof(T) % 8 == 0, "8-byte words");
  T v;
  const long long *s = reinterpret_cast<const long long *>(p);
  long long *d = reinterpret_cast<long long *>(&v);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(T) / 8); ++i) d[i] = __ldcg(s + i);
  return v;
}

enum : int { kClaimExit = 0, kClaimChain = 1, kClaimRefine = 2 };

struct Claim {
  int kind, slot, a, b, c;  // chain: a = job; refine: a = group, b = step, c = task
};

// Thread 0 of a CTA: the next job, or kClaimExit. Refinement tasks come first (they end
// requests already under way), then chain jobs of short requests, then of long ones.
__device__ Claim claim_next(const ResParams &p) {
  ResCtl *ctl = p.ctl;
  unsigned sleep_ns = 2000;
  int64_t empty = 0;
  for (int64_t polls = 0;; ++polls) {
    if (*(volatile int32_t *)&ctl->quit) return {kClaimExit, 0, 0, 0, 0};
    const unsigned long long dh = *(volatile unsigned long long *)&ctl->dhead;
    const unsigned long long dt = *(volatile unsigned long long *)&ctl->dtail;
    if (dh < dt) {
      if (atomicCAS(&ctl->dhead, dh, dh + 1) != dh) continue;
      atomicAdd(&ctl->busy, 1);
      ResTask *e = p.dring + (dh & p.dring_mask);
      const uint32_t want = (uint32_t)(dh + 1);
      int64_t w = 0;
      while (ld_acquire_u32(&e->seq) != want && ++w < kSeqWaitPolls) {
      }
      if (w >= kSeqWaitPolls) {  // the producer never released it: drop the entry
        atomicOr(p.err, kErrTimeout);
        atomicSub(&ctl->busy, 1);
        continue;
      }
      return {kClaimRefine, __ldcg(&e->slot), __ldcg(&e->group), __ldcg(&e->step), __ldcg(&e->task)};
    }
    // chain jobs: the ring of short requests first
    bool lost = false;
    for (int c = 0; c < 2 && !lost; ++c) {
      const unsigned long long h = *(volatile unsigned long long *)&ctl->head[c];
      const unsigned long long t = ld_acquire_u64(&ctl->tail[c]);
      if (h >= t) continue;
      if (atomicCAS(&ctl->head[c], h, h + 1) != h) {
        lost = true;  // another CTA took it: poll again from the top
        break;
      }
      atomicAdd(&ctl->busy, 1);
      const ResEntry *ring = p.ring + (unsigned long long)c * (p.ring_mask + 1);
      const int2 e = __ldcg(reinterpret_cast<const int2 *>(ring + (h & p.ring_mask)));
      return {kClaimChain, e.x, e.y, 0, 0};
    }
    if (lost) continue;
    // nothing to claim
    ++empty;
    const bool stop = *(volatile int32_t *)&ctl->stop != 0;
    if (stop || empty >= p.idle_polls || polls >= kIdleGiveUp) {
      // end the launch only when no CTA is busy and both rings are empty (busy first: a
      // job's refinement tasks are reserved before its CTA leaves `busy`)
      const int b = ld_acquire_i32(&ctl->busy);
      auto vol = [](const unsigned long long *q) { return *(const volatile unsigned long long *)q; };
      const bool empty_rings = vol(&ctl->dhead) == vol(&ctl->dtail) &&
                               vol(&ctl->head[0]) == ld_acquire_u64(&ctl->tail[0]) &&
                               vol(&ctl->head[1]) == ld_acquire_u64(&ctl->tail[1]);
      if ((b == 0 && empty_rings) || polls >= kIdleGiveUp) {
        atomicExch(&ctl->quit, 1);
        return {kClaimExit, 0, 0, 0, 0};
      }
    }
    __nanosleep(sleep_ns);
    if (sleep_ns < 32000) sleep_ns <<= 1;
  }
}

// Reserves and releases the refinement tasks of groups [g0, g1) of a request for `step`
// (all threads of the CTA call it).
__device__ void enqueue_refine(const ResParams &p, int slot, const ResItemDev &it, int g0, int g1, int step,
                               unsigned long long *s_base) {
  const int cnt = (g1 - g0) * it.nt;
  if (threadIdx.x == 0) *s_base = atomicAdd(&p.ctl->dtail, (unsigned long long)cnt);
  __syncthreads();
  const unsigned long long base = *s_base;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const unsigned long long idx = base + (unsigned long long)i;
    ResTask *e = p.dring + (idx & p.dring_mask);
    e->slot = slot;
    e->group = g0 + i / it.nt;
    e->step = step;
    e->task = i % it.nt;
    st_release_u32(&e->seq, (uint32_t)(idx + 1));
  }
  __syncthreads();
}

// The request in `slot` is complete: its status, then its sequence number, to the host.
__device__ void signal_done(const ResParams &p, int slot, const ResItemDev &it) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const int st = __ldcg(it.inst.status);
    __threadfence_system();
    *(volatile int32_t *)(p.hstatus + slot) = st;
    __threadfence_system();
    st_release_sys_i32(p.hdone + slot, it.seq);
  }
}

// A chain job of the request in `slot`, then every tree node it is the last child of (the
// batched kernel's climb), then, at the root, R and X or the first refinement step.
__device__ void run_chain(const ResParams &p, int slot, int jb, unsigned char *smraw, int *s_go,
                          unsigned long long *s_base) {
  const ResItemDev it = ldcg_struct(p.items + slot);
  const BatchInst &in = it.inst;
  for (;;) {
    const BatchJob bj = ldcg_struct(it.jobs + jb);
    const JobDesc jd{bj.piv_row, bj.tile_begin, bj.tile_count};
    const bool chain = jb < it.nchains;
    if (chain && in.mixed) {
      FactorParamsT<float> fp{};
      fp.A = in.A;
      fp.lda = in.lda;
      fp.V = static_cast<float *>(in.V);
      fp.ldv = in.ldv;
      fp.tiles = it.tiles;
      fp.tau = static_cast<float *>(in.tau);
      fp.scl = static_cast<float *>(in.scl);
      fp.n = in.n;
      fp.nc = in.n;
      fp.ldt = in.ldt;
      switch (in.n <= 16 ? 1 : (in.n <= 32 ? 2 : (in.n <= 64 ? 4 : 8))) {
        case 1: run_job_f32s<1, true>(fp, jd, smraw); break;
        case 2: run_job_f32s<2, true>(fp, jd, smraw); break;
        case 4: run_job_f32s<4, true>(fp, jd, smraw); break;
        default: run_job_f32s<8, true>(fp, jd, smraw); break;
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
      fp.tiles = it.tiles;
      fp.tau = chain ? static_cast<double *>(in.tau) : in.tau64;
      fp.scl = chain ? static_cast<double *>(in.scl) : in.scl64;
      fp.n = in.n;
      fp.nc = in.n + in.k;
      fp.ldt = chain ? in.ldt : in.ldt_tree;
      run_job<kResCmax, false, true>(fp, jd, smraw);
    }
    if (bj.parent < 0) {
      __threadfence();
      finish_instance(in, bj.row64, smraw);
      if (it.ngroups > 0)
        enqueue_refine(p, slot, it, 0, it.ngroups, 0, s_base);
      else
        signal_done(p, slot, it);
      return;
    }
    // publish this job's triangle, then arrive at the parent; the last child combines
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const int nchild = __ldcg(&it.jobs[bj.parent].nchild);
      *s_go = (atomicAdd(it.counters + bj.parent, 1) == nchild - 1);
    }
    __syncthreads();
    const int go = *s_go;
    __syncthreads();
    if (!go) return;
    __threadfence();
    jb = bj.parent;
  }
}

// One refinement task; the last task of its step either releases the next step's tasks of
// its group or, when the group has stopped, counts the group out (the last group out
// completes the request). s_dec: two words of shared memory (the task's decision and its
// arrival flag).
__device__ void run_refine(const ResParams &p, int slot, int group, int step, int task, unsigned char *smraw,
                           int *s_dec, unsigned long long *s_base) {
  const ResItemDev it = ldcg_struct(p.items + slot);
  const RefineInst in = ldcg_struct(it.rinst + group);
  RefineTask tk{};
  tk.row0 = (int64_t)task * p.refine_rows;
  tk.rows = (int32_t)((it.m - tk.row0) < p.refine_rows ? (it.m - tk.row0) : p.refine_rows);
  tk.inst = group;
  tk.idx = task;
  RefineParams rp{};
  rp.step = step;
  rp.max_steps = p.max_steps;
  rp.tol = p.tol;
  if (threadIdx.x == 0) *s_dec = 0;
  __syncthreads();
  const int tb = (in.n + 31) / 32;
#define TSQR_RES_REFINE_CASE(K, T) \
  case K * 8 + T: refine_task<K, T, true>(rp, tk, in, smraw, s_dec); break;
#define TSQR_RES_REFINE_K(K) \
  TSQR_RES_REFINE_CASE(K, 1) TSQR_RES_REFINE_CASE(K, 2) TSQR_RES_REFINE_CASE(K, 3) TSQR_RES_REFINE_CASE(K, 4)
  switch (in.kb * 8 + tb) {
    TSQR_RES_REFINE_K(1) TSQR_RES_REFINE_K(2) TSQR_RES_REFINE_K(3) TSQR_RES_REFINE_K(4)
    TSQR_RES_REFINE_K(5) TSQR_RES_REFINE_K(6) TSQR_RES_REFINE_K(7) TSQR_RES_REFINE_K(8)
    default: break;
  }
#undef TSQR_RES_REFINE_K
#undef TSQR_RES_REFINE_CASE
  __syncthreads();
  const int dec = *s_dec;
  if (dec == 1) {
    __threadfence();
    enqueue_refine(p, slot, it, group, group + 1, step + 1, s_base);
  } else if (dec == 2) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *s_dec = (atomicSub(it.pending, 1) == 1) ? 3 : 0;
    __syncthreads();
    if (*s_dec == 3) signal_done(p, slot, it);
  }
}

__global__ void __launch_bounds__(kThreads, 2) k_resident(const ResParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_kind, s_slot, s_a, s_b, s_c, s_go, s_dec[2];
  __shared__ unsigned long long s_base;
  for (;;) {
    if (threadIdx.x == 0) {
      const Claim c = claim_next(p);
      s_kind = c.kind;
      s_slot = c.slot;
      s_a = c.a;
      s_b = c.b;
      s_c = c.c;
    }
    __syncthreads();
    const int kind = s_kind, slot = s_slot, a = s_a, b = s_b, c = s_c;
    __syncthreads();
    if (kind == kClaimExit) return;
    if (kind == kClaimChain)
      run_chain(p, slot, a, smraw, &s_go, &s_base);
    else
      run_refine(p, slot, a, b, c, smraw, s_dec, &s_base);
    // leave `busy` after the job's enqueues are visible
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicSub(&p.ctl->busy, 1);
  }
}

}  // namespace

cudaError_t launch_resident(const ResParams &p, int grid, size_t smem_bytes, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_resident, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e != cudaSuccess) return e;
  k_resident<<<grid, kThreads, smem_bytes, s>>>(p);
  return cudaGetLastError();
}

}  // namespace tsqr
