// Bulk asynchronous copies (the TMA engine's untiled mode) from global to
// shared memory, completed on an mbarrier, with a bounded wait.
//
// Rules the callers keep: the global source and the shared destination start
// on 16-byte boundaries and the size is a multiple of 16 bytes (checked by the
// caller before every copy; a copy that does not meet them is not issued);
// one thread arms the barrier with the byte count and issues the copy; every
// waiter tracks the barrier's phase parity itself.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define PD_BULK_WAIT_NS 1000000000ull  // a wait gives up after one second
#define PD_BULK_WAIT_POLLS (1u << 24)  // ... or after this many polls

__device__ __forceinline__ uint32_t pd_smem(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void pd_mbar_init(uint64_t *bar, uint32_t arrivals) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(pd_smem(bar)), "r"(arrivals) : "memory");
}

// Makes initialised barriers visible to the copy engine (before first use).
__device__ __forceinline__ void pd_mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses before later bulk
// copies into the same words (generic proxy -> async proxy).
__device__ __forceinline__ void pd_fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One arrival that also expects `bytes` of copy transactions on the phase.
__device__ __forceinline__ void pd_mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(pd_smem(bar)), "r"(bytes)
               : "memory");
}

// `bytes` from global `src` to shared `dst`, counted on `bar` when they land.
__device__ __forceinline__ void pd_bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          pd_smem(dst)),
      "l"(src), "r"(bytes), "r"(pd_smem(bar))
      : "memory");
}

__device__ __forceinline__ bool pd_mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(pd_smem(bar)), "r"(parity)
      : "memory");
  return done != 0u;
}

__device__ __forceinline__ uint64_t pd_globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase of `bar` with parity `parity` to complete.  Returns
// false if it has not after PD_BULK_WAIT_NS nanoseconds or PD_BULK_WAIT_POLLS
// polls, whichever comes first.
__device__ __forceinline__ bool pd_mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  const uint64_t t0 = pd_globaltimer();
  for (uint32_t it = 0; it < PD_BULK_WAIT_POLLS; ++it) {
    if (pd_mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 63u && pd_globaltimer() - t0 > PD_BULK_WAIT_NS) return false;
  }
  return false;
}
