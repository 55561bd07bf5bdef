// Thread-block-cluster helpers: distributed shared memory addressing, st.async
// transfers that complete a receiver's mbarrier, bounded waits on those
// mbarriers and the cluster-wide barrier.  Used by the cluster triangular
// solve (k_tri.cu) and the blocked Householder QR (k_qr_blocked.cu).
#pragma once
#include "lsq_common.cuh"

namespace lsq {

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_nranks() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// the same shared-memory variable in CTA `rank` of the cluster
__device__ __forceinline__ unsigned cluster_addr(const void *p, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_async_f64(unsigned raddr, double v, unsigned rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(raddr),
               "l"(__double_as_longlong(v)), "r"(rbar)
               : "memory");
}
// An mbarrier for one transfer of `bytes`: its one arrival is made here, the
// phase completes when the remote stores have delivered the bytes.
__device__ __forceinline__ void xfer_bar_init(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// make the barrier initialisations visible to the cluster's remote arrivals
__device__ __forceinline__ void fence_mbarrier_init_cluster() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool xfer_try(uint64_t *bar) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar))
      : "memory");
  return ok != 0;
}
// wait for the transfer, giving up after limit_ns
__device__ __forceinline__ bool xfer_wait_limit(uint64_t *bar, uint64_t limit_ns) {
  if (xfer_try(bar)) return true;
  const uint64_t t0 = global_ns();
  while (!xfer_try(bar))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

}  // namespace lsq
