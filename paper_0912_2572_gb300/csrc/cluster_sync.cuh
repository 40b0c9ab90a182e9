// Thread-block cluster primitives shared by the cluster tier of the factorization and of
// the application of Q (sm_103a): distributed-shared-memory addressing (mapa), loads from a
// peer CTA's shared memory, progress counters published with release stores and read with
// acquire loads at cluster scope, and the cluster-wide barrier.
#pragma once
#include <cstdint>

namespace tsqr {

// polls of a peer's progress counter before a wait gives up (each poll sleeps at least
// 32 ns: above 0.1 s, five orders of magnitude above a column step)
constexpr uint32_t kClusterSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t cluster_map(uint32_t addr, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ uint32_t ld_acquire_cluster_u32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ double ld_cluster_f64(uint32_t addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_cluster_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.release.cluster.shared::cta.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ int cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}

}  // namespace tsqr
