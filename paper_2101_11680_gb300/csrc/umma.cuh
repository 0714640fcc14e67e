// tcgen05 (5th-generation tensor core) building blocks, inline PTX for
// sm_100a / sm_103a: shared-memory matrix descriptors for the no-swizzle
// K-major layout, the TF32 instruction descriptor, the MMA issue and its
// completion through an mbarrier, tensor-memory (TMEM) allocation, and the
// 32-lane TMEM loads and stores of the epilogues.  (The learned CNN's
// convolution ORs the 32-byte swizzle mode, 6, into bits 61-63 of a
// descriptor for its 32-byte operand rows; see learned.cu.)
//
// Operand layout used by the contractions (no swizzle, K-major): a tile of R rows
// (R a multiple of 8) and K FP32 columns (K a multiple of 4) stores element
// (r, k) at byte ((k / 4) * R + r) * 16 + (k % 4) * 4: for each group of four
// k, the R rows follow each other as 16-byte rows.  A core matrix (8 rows x
// 16 bytes) is then 128 contiguous bytes; core matrices adjacent in K are
// R * 16 bytes apart (the descriptor's leading-dimension byte offset) and
// those adjacent in rows 128 bytes apart (its stride-dimension byte offset).
// An MMA with K = 8 (TF32) reads two k-groups, so step s starts 2 s R 16
// bytes into the tile, and rows r0.. start r0 * 16 bytes in.
#pragma once
#include <cstdint>

namespace umma {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, leading (K-direction) and
// stride (row-direction) byte offsets, all in 16-byte units; bits 46-47 hold
// the descriptor version 1; swizzle mode 0 (none) in bits 61-63.
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32 with FP32 accumulation, both operands
// K-major: D format F32 (bits 4-5 = 1), A and B format TF32 (bits 7-9 and
// 10-12 = 2), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// D[tmem] (+)= A * B^T for one K = 8 step; accumulate = 0 overwrites D.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// The mbarrier completes one arrival when every tcgen05 operation this
// thread issued before has finished.
__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Wait until the phase with the given parity has completed; gives up after
// max_polls polls (returns false) so that a lost completion cannot hang the GPU.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, long long max_polls) {
  const uint32_t a = smem_u32(mbar);
  for (long long i = 0; i < max_polls; ++i) {
    uint32_t done;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Generic-proxy shared-memory writes -> visible to the tensor core's reads.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Warp-wide: allocate ncols (a power of two >= 32) TMEM columns; the base
// address lands in *dst (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

// Warp-wide: lane l of the warp reads 16 consecutive FP32 columns of TMEM
// lane (taddr >> 16) + l, starting at column taddr & 0xFFFF (the warp may only
// address the 32-lane quarter 32 (warp % 4) .. 32 (warp % 4) + 31).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Warp-wide: lane l writes r[0..7] to 8 consecutive 32-bit columns of TMEM
// lane (taddr >> 16) + l from column taddr & 0xFFFF (same lane quarter rule as
// tmem_ld16).  Complete (and visible to later tcgen05 operations of other
// threads) after tmem_wait_st and a fence_before_sync / barrier hand-off.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// Byte offset of element (r, k) in a K-major no-swizzle tile of `rows` rows.
__host__ __device__ constexpr uint32_t kmajor_off(int rows, int r, int k) {
  return (uint32_t)((((k >> 2) * rows + r) << 4) + ((k & 3) << 2));
}

// Split x = hi + lo with hi on the TF32 grid (round to nearest) and lo the
// exact FP32 remainder; three products hi*hi + hi*lo + lo*hi recover FP32
// accuracy on the TF32 tensor path.
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  lo = x - hi;
}

}  // namespace umma
