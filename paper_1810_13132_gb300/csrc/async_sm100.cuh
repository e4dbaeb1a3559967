// async_sm100.cuh -- inline-PTX wrappers for the asynchronous data movement
// of sm_100-class GPUs: mbarriers (arrive, expected transactions, bounded
// waits) and TMA bulk copies global -> shared that complete on an mbarrier.
// Used by the planned estimate (its register-chunk ring) and by the
// bounded-wait self-test.
#pragma once
#include <cstdint>

namespace vbk {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// One arrival that also expects `bytes` of asynchronous-copy transactions.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}
// TMA bulk copy global -> shared (16-byte aligned, a multiple of 16 bytes),
// completing its bytes on the mbarrier b.
__device__ __forceinline__ void bulk_load_g2s(void *dst, const void *src, uint32_t bytes,
                                             uint64_t *b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(b))
      : "memory");
}

// Wait for the completion of the phase of parity `parity`, parking the warp
// between polls; false after `limit_ns` of %globaltimer.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *b, uint32_t parity, uint64_t limit_ns) {
  auto poll = [&]() {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(b)), "r"(parity), "n"(20000)
        : "memory");
    return done != 0;
  };
  if (poll()) return true;
  uint64_t t0, t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t0));
  do {
    if (poll()) return true;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  } while (t - t0 < limit_ns);
  return false;
}

}  // namespace vbk
