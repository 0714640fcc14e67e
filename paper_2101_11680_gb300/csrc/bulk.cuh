// Bulk-copy (TMA engine) helpers: mbarrier-completed global -> shared copies
// and bulk-group shared -> global copies (PTX cp.async.bulk, sm_90 and later).
// Addresses and sizes of every copy are multiples of 16 bytes.  Internal
// header: not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bulk {

// Polls of the wait that follows a timed-out wait (copies still in flight).
constexpr long long DRAIN_POLLS = 1ll << 24;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// One-phase barrier for `count` arrivals; visible to the copy engine.
__device__ __forceinline__ void bar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Arrive and announce `bytes` of copies that complete on the barrier.
__device__ __forceinline__ void arrive_expect(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(saddr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for the phase with the given parity; gives up after max_polls polls.
__device__ __forceinline__ bool wait(uint64_t* bar, uint32_t parity, long long max_polls) {
  for (long long i = 0; i < max_polls; ++i)
    if (try_wait(bar, parity)) return true;
  return false;
}

// Global -> shared, completing `bytes` on bar.
__device__ __forceinline__ void g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(bar))
               : "memory");
}

// Shared -> global in the issuing thread's current bulk group.
__device__ __forceinline__ void s2g(void* dst, const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(saddr(src)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }

// Until the thread's committed shared -> global copies have read their source.
__device__ __forceinline__ void wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }

// Orders this thread's generic-proxy shared-memory writes before later bulk copies.
__device__ __forceinline__ void fence_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

}  // namespace bulk
