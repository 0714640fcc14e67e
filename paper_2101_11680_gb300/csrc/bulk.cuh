// Bulk-copy (TMA engine) helpers: mbarrier-completed global -> shared copies
// and bulk-group shared -> global copies (PTX cp.async.bulk and
// cp.async.bulk.tensor, sm_90 and later).  Addresses and sizes of every plain
// bulk copy are multiples of 16 bytes.  Internal header: not part of the C ABI.
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

// Block-wide wait: thread 0 polls (at most max_polls times) while the other
// threads sleep at the block barrier; after it each thread acquires the
// completed phase with one poll of its own.  True when the phase completed.
__device__ __forceinline__ bool block_wait(uint64_t* bar, uint32_t parity, long long max_polls) {
  int ok = 1;
  if (threadIdx.x == 0) ok = wait(bar, parity, max_polls) ? 1 : 0;
  ok = __syncthreads_and(ok);
  if (ok && threadIdx.x != 0) (void)try_wait(bar, parity);
  return ok != 0;
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

// Tensor-map (tiled) copies of a 3-D box at element coordinates (c0, c1, c2);
// `map` is the address of a __grid_constant__ CUtensorMap kernel parameter.
// c0 * element size must be a multiple of 16 bytes; out-of-range elements are
// zero-filled on loads and skipped on stores.
__device__ __forceinline__ void tensor_g2s(void* dst, const void* map, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ void tensor_g2s_4d(void* dst, const void* map, int c0, int c1, int c2, int c3,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];\n" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ void tensor_g2s_5d(void* dst, const void* map, int c0, int c1, int c2, int c3, int c4,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5, %6}], [%7];\n" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ void tensor_g2s_2d(void* dst, const void* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];\n" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(saddr(bar))
      : "memory");
}

// Plain arrival (one of the barrier's expected arrivals).
__device__ __forceinline__ void arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ void tensor_s2g(const void* map, int c0, int c1, int c2, const void* src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(c0), "r"(c1), "r"(c2), "r"(saddr(src))
               : "memory");
}

__device__ __forceinline__ void commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }

// Until all but the N most recent of the thread's committed shared -> global
// bulk groups have read their source.
template <int N>
__device__ __forceinline__ void wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
}

// Orders this thread's generic-proxy shared-memory writes before later bulk copies.
__device__ __forceinline__ void fence_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

}  // namespace bulk
