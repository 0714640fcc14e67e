// Precision form: Tikhonov reconstruction of a batch of B measurement volumes
// that share one kernel (the per-frequency regularised inverse of Eq. 7 for
// B measurements at once), with the per-frequency contraction
// b = W_hat^T m_hat on the 5th-generation tensor cores in BF16 or FP8 (e4m3)
// and the Z x Z solve refined iteratively:
//
//   b0 = first product term only,  b = all product terms (FP32 accumulation)
//   x0 = C b0,   x_{i+1} = x_i + C (b - (G + lambda I) x_i)
//
// with C = (G + lambda I)^-1 (FP64 Cholesky) and G the FP64 Gram.  Operands
// are split into narrow-format terms whose sum reproduces the FP32 value:
//
//   BF16: v = v_hi + v_lo (both BF16); b0 = hi.hi, b = hi.hi + (hi.lo + lo.hi)
//   FP8:  v = s (q0 + q1/16 + q2/256), each q an e4m3 value, s a scale that
//         maps the block's largest magnitude to 448 (per frequency class for
//         W_hat, per right-hand side for m_hat); products grouped by level:
//         D0 = q0.p0, D1 = q0.p1 + q1.p0, D2 = q0.p2 + q1.p1 + q2.p0,
//         b0 = s_w s_m D0,  b = s_w s_m (D0 + D1/16 + D2/256)
//
// (a 2-term e4m3 split leaves the refined solution ~1e-2 from the exact one
// on small grids; three terms bring it to ~1e-4).  The solve's products
// (C b0, (G + lambda I) x, C r) run on the same tensor cores in TF32 with
// hi/lo splits of both operands (three products each: FP32-level results):
// the residual b - (G + lambda I) x is a small difference of nearly equal
// terms, and BF16-level products there left the refined result at ~2e-4.
//
// One CTA of 8 warps per SM walks the frequency classes.  Per class, the
// tables C and G + lambda I (BF16 hi/lo, canonical K-major layout, made once
// per lambda, TF32 hi/lo) come in with 16-byte cp.async copies; the batch is taken 16 volumes at a
// time: 16 volumes x 4 members x re/im = 128 right-hand sides = the M side of
// the GEMM D[n][z] = sum_t m[n][t] W[t][z] (M = 128, N = Z rounded up to 16,
// K = t in chunks of 32).  Each t chunk of m_hat rows and W_hat rows streams
// into a ring of four raw shared-memory stages with cp.async copies, three
// chunks ahead of the one being split into its terms (W^T read down padded
// columns) and multiplied; the term buffers are double-buffered as well,
// each set guarded by its own MMA-completion mbarrier.  After the last chunk
// the refinement runs on the TMEM accumulators: each thread owns one
// right-hand side (a TMEM lane) and half of its Z columns.  Every wait is
// bounded; a wait that runs out sets the handle's sticky flag, drains the
// MMAs in flight and stops the CTA.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "bulk.cuh"
#include "ctof_internal.h"
#include "umma.cuh"

namespace {

constexpr int BT_THREADS = 256;
constexpr int VB = 16;             // volumes per chunk
constexpr int NR = 8 * VB;         // right-hand sides per chunk (the GEMM's M = 128)
constexpr int TCH = 32;            // t values per K chunk
constexpr int RCS = TCH * 8 + 8;   // raw stage bytes per (volume, member) row: 66 words, rows 2 banks apart
constexpr int RAW_STAGES = 4;      // raw copies run this many t chunks ahead, minus one
constexpr long long DRAIN_POLLS = 1ll << 24;
constexpr float E4M3_MAX = 448.f;

inline int rup(int x, int m) { return (x + m - 1) / m * m; }

struct BtPlan {
  int nt, nz, z4, zn;  // zn = nz rounded up to 16 (N of the GEMMs, K of the solve)
  int fp8, nterm, esize, epc;  // epc = elements per 16-byte core-matrix row
  int a_term, b_term;          // bytes of one term of the A (m) and B (W^T) chunk tiles
  int set_bytes;               // A terms + B terms
  int raw_c, raw_stage;
  int tab_bytes;               // C hi, C lo, G' hi, G' lo (TF32, zn x zn each)
  int x_tile;                  // one TF32 [128][zn] A operand of the solve
  int off_set, off_raw, off_tab, off_xh, off_xl, off_sn, off_bar, total;
  int batch;
};

BtPlan make_plan(int nt, int nz, int fp8, int batch) {
  BtPlan P{};
  P.nt = nt;
  P.nz = nz;
  P.z4 = rup(nz, 4);
  P.zn = rup(nz, 16);
  P.fp8 = fp8;
  P.nterm = fp8 ? 3 : 2;
  P.esize = fp8 ? 1 : 2;
  P.epc = 16 / P.esize;
  P.a_term = NR * TCH * P.esize;
  P.b_term = P.zn * TCH * P.esize;
  P.set_bytes = P.nterm * (P.a_term + P.b_term);
  P.raw_c = rup(4 * VB * RCS, 16);
  P.raw_stage = P.raw_c + TCH * (P.z4 + 4) * 4;  // W rows padded by 4 floats: column reads on distinct banks
  P.tab_bytes = 4 * P.zn * P.zn * 4;
  P.x_tile = NR * P.zn * 4;
  P.batch = batch;
  int off = 0;
  auto take = [&](int bytes) {
    const int at = off;
    off += rup(bytes, 128);
    return at;
  };
  P.off_set = take(2 * P.set_bytes);
  P.off_raw = take(RAW_STAGES * P.raw_stage);
  P.off_tab = take(P.tab_bytes);
  // the solve's operands reuse the term sets and raw stages (idle by then)
  P.off_xh = P.off_set;
  P.off_xl = P.off_set + rup(P.x_tile, 128);
  P.off_sn = take(NR * 4);
  P.off_bar = take(64);
  P.total = off;
  return P;
}

// Instruction descriptors (FP32 accumulation, both operands K-major): D format
// F32 in bits 4-5, A / B formats in bits 7-9 / 10-12 (kind::f16: BF16 = 1;
// kind::f8f6f4: E4M3 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_e4m3(int m, int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_e4m3(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// Byte offset of the 16-byte core-matrix row holding elements (r, k .. k + epc - 1)
// of a K-major no-swizzle tile of `rows` rows (k a multiple of epc).
__device__ __forceinline__ uint32_t kchunk(int rows, int r, int k, int epc) {
  return (uint32_t)(((k / epc) * rows + r) << 4);
}

__device__ __forceinline__ unsigned pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<unsigned*>(&h);
}

// BF16 split of 8 values into hi / lo 16-byte rows.
__device__ __forceinline__ void split8_bf16(const float (&v)[8], uint4& hi, uint4& lo) {
  unsigned h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const float2 back = __bfloat1622float2(p);
    h[i] = *reinterpret_cast<const unsigned*>(&p);
    l[i] = pack_bf16x2(v[2 * i] - back.x, v[2 * i + 1] - back.y);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// e4m3 pair (round to nearest, saturating) and its value.
__device__ __forceinline__ unsigned short e4m3x2(float a, float b, float2& back) {
  const __nv_fp8x2_storage_t q = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(q, __NV_E4M3);
  back = __half22float2(*reinterpret_cast<const __half2*>(&hr));
  return (unsigned short)q;
}

// FP8 three-term split of 16 values already divided by their scale
// (|v| <= 448): v ~ q0 + q1/16 + q2/256.
__device__ __forceinline__ void split16_e4m3(const float (&v)[16], uint4& t0, uint4& t1, uint4& t2) {
  unsigned w0[4], w1[4], w2[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    unsigned a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const float x = v[4 * i + 2 * j], y = v[4 * i + 2 * j + 1];
      float2 b0, b1, b2;
      const unsigned short q0 = e4m3x2(x, y, b0);
      const float rx = x - b0.x, ry = y - b0.y;
      const unsigned short q1 = e4m3x2(16.f * rx, 16.f * ry, b1);
      const unsigned short q2 = e4m3x2(256.f * (rx - b1.x * 0.0625f), 256.f * (ry - b1.y * 0.0625f), b2);
      a0 |= (unsigned)q0 << (16 * j);
      a1 |= (unsigned)q1 << (16 * j);
      a2 |= (unsigned)q2 << (16 * j);
    }
    w0[i] = a0;
    w1[i] = a1;
    w2[i] = a2;
  }
  t0 = make_uint4(w0[0], w0[1], w0[2], w0[3]);
  t1 = make_uint4(w1[0], w1[1], w1[2], w1[3]);
  t2 = make_uint4(w2[0], w2[1], w2[2], w2[3]);
}

__device__ __forceinline__ void cp_async16z(void* smem, const void* gmem, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(umma::smem_u32(smem)), "l"(gmem), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async8z(void* smem, const void* gmem, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(umma::smem_u32(smem)), "l"(gmem), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_ahead() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(RAW_STAGES - 1) : "memory");
}
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ int pick(const int (&mem)[4], int m) {
  return m == 0 ? mem[0] : (m == 1 ? mem[1] : (m == 2 ? mem[2] : mem[3]));
}

// Raw copies of one t chunk: 64 (volume, member) rows of TCH complex m_hat
// values (8-byte copies: rows RCS bytes apart) and TCH rows of W_hat (16-byte
// copies, rows z4 + 4 floats apart); zero fill beyond nt, for absent members
// and for v >= nv.
__device__ __forceinline__ void issue_raw(const BtPlan& P, unsigned char* raw, const int (&mem)[4], int v0, int nv,
                                          int t0, const float* __restrict__ wc, const float2* __restrict__ m_hat,
                                          int ldm) {
  const int nt = P.nt;
  for (int i = threadIdx.x; i < 4 * VB * TCH; i += BT_THREADS) {
    const int vm = i / TCH, p = i - vm * TCH;
    const int v = vm >> 2, f = pick(mem, vm & 3), t = t0 + p;
    const int bytes = (f < 0 || v >= nv || t >= nt) ? 0 : 8;
    const float2* src = bytes ? m_hat + (size_t)f * ldm + (size_t)(v0 + v) * nt + t : m_hat;
    cp_async8z(raw + vm * RCS + p * 8, src, bytes);
  }
  unsigned char* rw = raw + P.raw_c;
  const int q4 = P.z4 >> 2, ws = P.z4 + 4;
  for (int i = threadIdx.x; i < TCH * q4; i += BT_THREADS) {
    const int tl = i / q4, k4 = i - tl * q4, t = t0 + tl;
    const int bytes = t < nt ? 16 : 0;
    cp_async16z(rw + (tl * ws + 4 * k4) * 4, bytes ? wc + (size_t)t * P.z4 + 4 * k4 : wc, bytes);
  }
}

// Split the raw chunk into its terms: A = m rows (n = 8 v + 2 member + re/im,
// K = t), B = W^T rows (z, K = t).  s_n: per right-hand-side scales (FP8).
// A item = (volume-member row, group of epc t): one float2 read per t gives
// both the real (row 2 vm) and imaginary (row 2 vm + 1) right-hand sides;
// B item = (z, group of epc t), read down a padded W column.  Consecutive
// threads take consecutive rows, so reads and 16-byte term stores hit
// distinct banks.
__device__ __forceinline__ void convert_chunk(const BtPlan& P, const unsigned char* raw, unsigned char* set,
                                              const float* s_n, float inv_sw) {
  const int epc = P.epc, groups = TCH / epc;
  unsigned char* a = set;                       // nterm A terms
  unsigned char* b = set + P.nterm * P.a_term;  // nterm B terms
  for (int i = threadIdx.x; i < 4 * VB * groups; i += BT_THREADS) {
    const int vm = i & (4 * VB - 1), gI = i / (4 * VB);
    const float2* row = reinterpret_cast<const float2*>(raw + vm * RCS) + gI * epc;
    const uint32_t o_re = kchunk(NR, 2 * vm, gI * epc, epc), o_im = kchunk(NR, 2 * vm + 1, gI * epc, epc);
    if (P.fp8) {
      const float sr = 1.f / s_n[2 * vm], si = 1.f / s_n[2 * vm + 1];
      float vr[16], vi[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const float2 x = row[e];
        vr[e] = x.x * sr;
        vi[e] = x.y * si;
      }
      uint4 t0, t1, t2;
      split16_e4m3(vr, t0, t1, t2);
      *reinterpret_cast<uint4*>(a + o_re) = t0;
      *reinterpret_cast<uint4*>(a + P.a_term + o_re) = t1;
      *reinterpret_cast<uint4*>(a + 2 * P.a_term + o_re) = t2;
      split16_e4m3(vi, t0, t1, t2);
      *reinterpret_cast<uint4*>(a + o_im) = t0;
      *reinterpret_cast<uint4*>(a + P.a_term + o_im) = t1;
      *reinterpret_cast<uint4*>(a + 2 * P.a_term + o_im) = t2;
    } else {
      float vr[8], vi[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float2 x = row[e];
        vr[e] = x.x;
        vi[e] = x.y;
      }
      uint4 hi, lo;
      split8_bf16(vr, hi, lo);
      *reinterpret_cast<uint4*>(a + o_re) = hi;
      *reinterpret_cast<uint4*>(a + P.a_term + o_re) = lo;
      split8_bf16(vi, hi, lo);
      *reinterpret_cast<uint4*>(a + o_im) = hi;
      *reinterpret_cast<uint4*>(a + P.a_term + o_im) = lo;
    }
  }
  // B rows z in [z4, zn) stay zero: the solve's operands share this memory
  for (int i = threadIdx.x; i < (P.zn - P.z4) * groups; i += BT_THREADS) {
    const int z = P.z4 + i % (P.zn - P.z4), gI = i / (P.zn - P.z4);
    const uint32_t o = kchunk(P.zn, z, gI * epc, epc);
    for (int tI = 0; tI < P.nterm; ++tI) *reinterpret_cast<uint4*>(b + tI * P.b_term + o) = make_uint4(0u, 0u, 0u, 0u);
  }
  const float* rw = reinterpret_cast<const float*>(raw + P.raw_c);
  const int ws = P.z4 + 4;
  for (int i = threadIdx.x; i < P.z4 * groups; i += BT_THREADS) {
    const int z = i % P.z4, gI = i / P.z4;
    const float* col = rw + gI * epc * ws + z;
    const uint32_t o = kchunk(P.zn, z, gI * epc, epc);
    if (P.fp8) {
      float w[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) w[e] = col[e * ws] * inv_sw;
      uint4 t0, t1, t2;
      split16_e4m3(w, t0, t1, t2);
      *reinterpret_cast<uint4*>(b + o) = t0;
      *reinterpret_cast<uint4*>(b + P.b_term + o) = t1;
      *reinterpret_cast<uint4*>(b + 2 * P.b_term + o) = t2;
    } else {
      float w[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) w[e] = col[e * ws];
      uint4 hi, lo;
      split8_bf16(w, hi, lo);
      *reinterpret_cast<uint4*>(b + o) = hi;
      *reinterpret_cast<uint4*>(b + P.b_term + o) = lo;
    }
  }
}

// Bounded wait on an MMA-completion mbarrier (block-wide: true = some thread
// gave up; then every thread has drained and the CTA must stop).
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t& phase, int* flag, long long max_polls) {
  int gave_up = 0;
  if (!umma::mbar_wait(bar, phase, max_polls)) {
    gave_up = 1;
    atomicExch(flag, 1);
    umma::mbar_wait(bar, phase, DRAIN_POLLS);
  }
  phase ^= 1u;
  umma::fence_after_sync();
  return __syncthreads_or(gave_up) != 0;
}

__device__ __forceinline__ void publish() {
  umma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
}

// Three TF32 products D (+)= X_lo T_hi + X_hi T_lo + X_hi T_hi of the solve:
// X = [128][zn] (A, K = w), T = table rows z (B, K = w).
__device__ __forceinline__ void issue_solve3(uint32_t d, uint32_t xh, uint32_t xl, uint32_t th, uint32_t tl, int zn) {
  const uint32_t idesc = umma::idesc_tf32(NR, zn);
  for (int s = 0; s < zn / 8; ++s) {
    const uint32_t oa = s * 2 * NR * 16, ob = s * 2 * zn * 16;
    const uint64_t ah = umma::desc(xh + oa, NR * 16, 128), al = umma::desc(xl + oa, NR * 16, 128);
    const uint64_t bh = umma::desc(th + ob, zn * 16, 128), bl = umma::desc(tl + ob, zn * 16, 128);
    umma::mma_tf32(d, al, bh, idesc, s > 0);
    umma::mma_tf32(d, ah, bl, idesc, 1);
    umma::mma_tf32(d, ah, bh, idesc, 1);
  }
}

// Row n of the solve operand X (K = w): TF32 hi / lo of 16 values at w = 16 j.
__device__ __forceinline__ void put_x16(unsigned char* xh, unsigned char* xl, int n, int j, const float (&v)[16]) {
#pragma unroll
  for (int qd = 0; qd < 4; ++qd) {
    float4 h, l;
    umma::split_tf32(v[4 * qd + 0], h.x, l.x);
    umma::split_tf32(v[4 * qd + 1], h.y, l.y);
    umma::split_tf32(v[4 * qd + 2], h.z, l.z);
    umma::split_tf32(v[4 * qd + 3], h.w, l.w);
    const uint32_t o = kchunk(NR, n, 16 * j + 4 * qd, 4);
    *reinterpret_cast<float4*>(xh + o) = h;
    *reinterpret_cast<float4*>(xl + o) = l;
  }
}

__global__ void __launch_bounds__(BT_THREADS, 1) k_batch_tikhonov_tc(
    BtPlan P, const float* __restrict__ what, const unsigned char* __restrict__ tabs,
    const float* __restrict__ class_scale, const int* __restrict__ members, int nclass,
    const float2* __restrict__ m_hat, int ldm, float2* __restrict__ x_hat, int ldx, int refine, int* flag,
    long long max_polls) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nt = P.nt, nz = P.nz, zn = P.zn;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + P.off_bar);  // [0], [1]: term sets; [2]: solve
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + P.off_bar + 32);
  float* s_n = reinterpret_cast<float*>(sm + P.off_sn);
  for (int i = tid; i < P.off_bar / 16; i += BT_THREADS)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < NR; i += BT_THREADS) s_n[i] = 1.f;
  __syncthreads();
  if (warp == 0) umma::tmem_alloc(tslot, 256);
  if (tid == 0) {
    umma::mbar_init(bars + 0, 1);
    umma::mbar_init(bars + 1, 1);
    umma::mbar_init(bars + 2, 1);
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t taddr = *tslot;
  uint32_t ph[3] = {0u, 0u, 0u};
  int pend[2] = {0, 0};  // commits on the term-set barriers not yet waited for
  const uint32_t sbase = umma::smem_u32(sm);
  const uint32_t col_acc0 = 0, col_acc1 = zn, col_acc2 = 2 * zn, col_work = 3 * zn;
  const uint32_t idesc_main = P.fp8 ? idesc_e4m3(NR, zn) : idesc_bf16(NR, zn);
  const int nchunks = (nt + TCH - 1) / TCH;
  const int nvc = (P.batch + VB - 1) / VB;
  // epilogue mapping: TMEM lane = right-hand side n, warps w and w + 4 take alternate 16-column groups
  const int q = warp & 3, half = warp >> 2, n = 32 * q + lane;
  const uint32_t trow = taddr + ((uint32_t)(32 * q) << 16);
  unsigned char* xh = sm + P.off_xh;
  unsigned char* xl = sm + P.off_xl;
  // solve tables in shared memory: C hi, C lo, G' hi, G' lo
  const uint32_t t_ch = sbase + P.off_tab, t_cl = t_ch + zn * zn * 4, t_gh = t_cl + zn * zn * 4,
                 t_gl = t_gh + zn * zn * 4;
  bool stop = false;
  for (int c = blockIdx.x; c < nclass && !stop; c += gridDim.x) {
    int mem[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) mem[m] = __ldg(members + 4 * c + m);
    const float* wc = what + (size_t)c * nt * P.z4;
    const float sw = P.fp8 ? __ldg(class_scale + c) : 1.f;
    const float inv_sw = 1.f / sw;
    // the class's solve tables (previous readers, the solve MMAs, have completed)
    {
      const uint4* src = reinterpret_cast<const uint4*>(tabs + (size_t)c * P.tab_bytes);
      for (int i = tid; i < P.tab_bytes / 16; i += BT_THREADS) cp_async16z(sm + P.off_tab + 16 * i, src + i, 16);
      cp_commit();
    }
    for (int vc = 0; vc < nvc && !stop; ++vc) {
      const int v0 = vc * VB, nv = P.batch - v0 < VB ? P.batch - v0 : VB;
      if (P.fp8) {
        // per right-hand-side scale: the largest magnitude over t maps to 448
        const int vm = tid >> 2, part = tid & 3, v = vm >> 2, f = pick(mem, vm & 3);
        float mr = 0.f, mi = 0.f;
        if (f >= 0 && v < nv) {
          const float2* src = m_hat + (size_t)f * ldm + (size_t)(v0 + v) * nt;
          for (int t = part; t < nt; t += 4) {
            const float2 x = __ldg(src + t);
            mr = fmaxf(mr, fabsf(x.x));
            mi = fmaxf(mi, fabsf(x.y));
          }
        }
        mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, 1));
        mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, 2));
        mi = fmaxf(mi, __shfl_xor_sync(0xffffffffu, mi, 1));
        mi = fmaxf(mi, __shfl_xor_sync(0xffffffffu, mi, 2));
        if (part == 0) {
          s_n[2 * vm] = mr > 0.f ? mr / E4M3_MAX : 1.f;
          s_n[2 * vm + 1] = mi > 0.f ? mi / E4M3_MAX : 1.f;
        }
        __syncthreads();
      }
      for (int kc = 0; kc < RAW_STAGES - 1; ++kc) {
        if (kc < nchunks) issue_raw(P, sm + P.off_raw + kc * P.raw_stage, mem, v0, nv, kc * TCH, wc, m_hat, ldm);
        cp_commit();
      }
      for (int kc = 0; kc < nchunks; ++kc) {
        const int ahead = kc + RAW_STAGES - 1;
        if (ahead < nchunks)
          issue_raw(P, sm + P.off_raw + (ahead % RAW_STAGES) * P.raw_stage, mem, v0, nv, ahead * TCH, wc, m_hat,
                    ldm);
        cp_commit();
        cp_wait_ahead();  // chunk kc has landed
        __syncthreads();
        const int set = kc & 1;
        if (pend[set]) {  // the MMAs that last read this term set
          if (wait_bar(bars + set, ph[set], flag, max_polls)) {
            stop = true;
            break;
          }
          pend[set] = 0;
        }
        unsigned char* sb = sm + P.off_set + set * P.set_bytes;
        convert_chunk(P, sm + P.off_raw + (kc % RAW_STAGES) * P.raw_stage, sb, s_n, inv_sw);
        publish();
        if (tid == 0) {
          const uint32_t a0 = sbase + P.off_set + set * P.set_bytes;
          const uint32_t b0 = a0 + P.nterm * P.a_term;
          const int ksteps = TCH * P.esize / 32;  // K steps of 32 bytes per row
          for (int s = 0; s < ksteps; ++s) {
            const uint32_t oa = s * 2 * NR * 16, ob = s * 2 * zn * 16;
            uint64_t A[3], B[3];
            for (int i = 0; i < P.nterm; ++i) {
              A[i] = umma::desc(a0 + i * P.a_term + oa, NR * 16, 128);
              B[i] = umma::desc(b0 + i * P.b_term + ob, zn * 16, 128);
            }
            const uint32_t first = (kc > 0 || s > 0) ? 1u : 0u;
            if (P.fp8) {
              mma_e4m3(taddr + col_acc0, A[0], B[0], idesc_main, first);
              mma_e4m3(taddr + col_acc1, A[0], B[1], idesc_main, first);
              mma_e4m3(taddr + col_acc1, A[1], B[0], idesc_main, 1);
              mma_e4m3(taddr + col_acc2, A[0], B[2], idesc_main, first);
              mma_e4m3(taddr + col_acc2, A[1], B[1], idesc_main, 1);
              mma_e4m3(taddr + col_acc2, A[2], B[0], idesc_main, 1);
            } else {
              mma_bf16(taddr + col_acc0, A[0], B[0], idesc_main, first);
              mma_bf16(taddr + col_acc1, A[0], B[1], idesc_main, first);
              mma_bf16(taddr + col_acc1, A[1], B[0], idesc_main, 1);
            }
          }
          umma::commit(bars + set);
        }
        pend[set] = 1;
      }
      if (stop) break;
      // all products of this chunk of volumes: wait for both term sets' last commits
      for (int s = 0; s < 2 && !stop; ++s) {
        if (pend[s]) {
          if (wait_bar(bars + s, ph[s], flag, max_polls)) stop = true;
          pend[s] = 0;
        }
      }
      if (stop) break;
      cp_wait0();  // the class tables
      __syncthreads();
      // ---- solve: x0 = C b0, then `refine` steps x += C (b - G' x) ----
      const float sn = s_n[n] * sw;
      float x[2][16];
      // b0 -> X
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        const int j = half + 2 * jj;
        if (16 * j < zn) {
          float v[16];
          umma::tmem_ld16(trow + col_acc0 + 16 * j, v);
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] *= P.fp8 ? sn : 1.f;
          put_x16(xh, xl, n, j, v);
        }
      }
      publish();
      if (tid == 0) {
        issue_solve3(taddr + col_work, sbase + P.off_xh, sbase + P.off_xl, t_ch, t_cl, zn);
        umma::commit(bars + 2);
      }
      if (wait_bar(bars + 2, ph[2], flag, max_polls)) {
        stop = true;
        break;
      }
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        const int j = half + 2 * jj;
        if (16 * j < zn) umma::tmem_ld16(trow + col_work + 16 * j, x[jj]);
      }
      for (int it = 0; it < refine && !stop; ++it) {
        // r = b - G' x
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int j = half + 2 * jj;
          if (16 * j < zn) put_x16(xh, xl, n, j, x[jj]);
        }
        publish();
        if (tid == 0) {
          issue_solve3(taddr + col_work, sbase + P.off_xh, sbase + P.off_xl, t_gh, t_gl, zn);
          umma::commit(bars + 2);
        }
        if (wait_bar(bars + 2, ph[2], flag, max_polls)) {
          stop = true;
          break;
        }
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int j = half + 2 * jj;
          if (16 * j < zn) {
            float gx[16], d0[16], d1[16], d2[16];
            umma::tmem_ld16(trow + col_work + 16 * j, gx);
            umma::tmem_ld16(trow + col_acc0 + 16 * j, d0);
            umma::tmem_ld16(trow + col_acc1 + 16 * j, d1);
            if (P.fp8) umma::tmem_ld16(trow + col_acc2 + 16 * j, d2);
            float r[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const float b = P.fp8 ? sn * (d0[e] + 0.0625f * d1[e] + 0.00390625f * d2[e]) : d0[e] + d1[e];
              r[e] = b - gx[e];
            }
            put_x16(xh, xl, n, j, r);
          }
        }
        // x += C r
        publish();
        if (tid == 0) {
          issue_solve3(taddr + col_work, sbase + P.off_xh, sbase + P.off_xl, t_ch, t_cl, zn);
          umma::commit(bars + 2);
        }
        if (wait_bar(bars + 2, ph[2], flag, max_polls)) {
          stop = true;
          break;
        }
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int j = half + 2 * jj;
          if (16 * j < zn) {
            float cr[16];
            umma::tmem_ld16(trow + col_work + 16 * j, cr);
#pragma unroll
            for (int e = 0; e < 16; ++e) x[jj][e] += cr[e];
          }
        }
      }
      if (stop) break;
      // x_hat[f][v * nz + z]: right-hand side n = 8 v + 2 member + re/im; even lanes write (re, im)
      {
        const int v = n >> 3, fm = pick(mem, (n >> 1) & 3);
        const bool writer = (lane & 1) == 0 && v < nv && fm >= 0;
        float2* dst = x_hat + (size_t)(fm >= 0 ? fm : 0) * ldx + (size_t)(v0 + (v < nv ? v : 0)) * nz;
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int j = half + 2 * jj;
          if (16 * j < zn) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const float im = __shfl_down_sync(0xffffffffu, x[jj][e], 1);
              const int z = 16 * j + e;
              if (writer && z < nz) dst[z] = make_float2(x[jj][e], im);
            }
          }
        }
      }
      // TMEM reads of this epilogue before the next chunk's MMAs overwrite the accumulators
      umma::fence_before_sync();
      __syncthreads();
    }
  }
  if (stop) {  // no MMA may still write TMEM when it is freed
    if (tid == 0) umma::commit(bars + 2);
    umma::mbar_wait(bars + 2, ph[2], DRAIN_POLLS);
  }
  cp_wait0();
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(taddr, 256);
}

// ======================= warp-specialised kernel (nt a multiple of 16) =======================
//
// Roles (14 warps): warp 0 (one thread) stages each chunk of TC t values with
// tensor-map copies (per member one m_hat box of TC/16 halves x 16 volumes x
// 16 t, W_hat boxes of TC t x 32 z, both in the 128-byte swizzle) into NS raw
// stages (TC = 32; NS = 2 at 64 depths, where shared memory holds no more;
// 16-t chunks with four stages measured slower: the hand-offs per chunk
// dominate); warps 1-8
// split a staged chunk into its narrow-format terms (NS term sets); warp 9 (one
// thread) issues the tcgen05 MMAs of each term set into one of two TMEM
// accumulator sets; warps 10-13 run the solve and the refinement of one
// (class, volume chunk) item from its accumulator set while the next item
// streams through the others.  Hand-offs go through mbarriers (raw full /
// empty, term full / empty, accumulators full / empty, class tables, solve
// MMAs); every wait is bounded, a wait that runs out sets the handle's flag
// and a shared abort word, and every role then leaves its loop.
// GEMM rows: right-hand side n = 32 member + 16 re/im + volume.

constexpr int WS_CONV = 8;      // converter warps 1 .. 8
constexpr int WS_MMA_WARP = 9;  // MMA issuer
constexpr int WS_EPI0 = 10;     // epilogue warps 10 .. 13
constexpr int WS_EPI = 4;
constexpr int WS_THREADS = (WS_EPI0 + WS_EPI) * 32;
constexpr int WS_MBOX = 16 * 16 * 8;  // m_hat box: 16 volumes x 16 t x 8 bytes
constexpr int WS_WBOX = 32 * 32 * 4;  // W_hat box: 32 t x 32 z x 4 bytes

struct WsPlan {
  int nt, nz, z4, zn, fp8, nterm, nacc, esize, epc;
  int tc, ns;     // t values per chunk, raw stages = term sets
  int a_term, b_term, set_bytes;
  int nwb;        // W boxes per chunk
  int raw_stage;  // bytes of one raw stage (1024-byte multiple)
  int tab_bytes, x_tile;
  int off_raw, off_set, off_tab, off_xh, off_xl, off_sn, off_bar, total;
  int batch, nvc;
};

WsPlan make_ws_plan(int nt, int nz, int fp8, int batch) {
  WsPlan P{};
  P.nt = nt;
  P.nz = nz;
  P.z4 = rup(nz, 4);
  P.zn = rup(nz, 16);
  P.fp8 = fp8;
  P.nterm = fp8 ? 3 : 2;
  P.nacc = fp8 ? 3 : 2;
  P.esize = fp8 ? 1 : 2;
  P.epc = 16 / P.esize;
  P.tc = 32;
  P.a_term = NR * P.tc * P.esize;
  P.b_term = P.zn * P.tc * P.esize;
  P.set_bytes = P.nterm * (P.a_term + P.b_term);
  P.nwb = P.z4 <= 32 ? 1 : 2;
  P.raw_stage = rup(4 * (P.tc / 16) * WS_MBOX + P.nwb * 32 * P.tc * 4, 1024);
  P.tab_bytes = 4 * P.zn * P.zn * 4;
  P.x_tile = NR * P.zn * 4;
  P.batch = batch;
  P.nvc = (batch + VB - 1) / VB;
  for (P.ns = 4; P.ns >= 2; --P.ns) {  // the deepest pipeline that fits
    int off = 0;
    auto take = [&](int bytes, int align) {
      off = rup(off, align);
      const int at = off;
      off += bytes;
      return at;
    };
    P.off_raw = take(P.ns * P.raw_stage, 1024);
    P.off_set = take(P.ns * P.set_bytes, 128);
    P.off_tab = take(P.tab_bytes, 128);
    P.off_xh = take(P.x_tile, 128);
    P.off_xl = take(P.x_tile, 128);
    P.off_sn = take(2 * NR * 4, 16);
    P.off_bar = take(512, 16);
    P.total = off + 1024;  // room to align the dynamic shared memory base to 1024 bytes
    if (P.total <= 227 * 1024) break;
  }
  return P;
}

__device__ __forceinline__ int ws_row(int v, int m, int ri) { return 32 * m + 16 * ri + v; }

// Bounded wait that also stops once another role has given up; after a few
// polls it sleeps between polls so that waiting warps leave the issue slots
// to the working ones.
__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t parity, long long max_polls, volatile int* abort_w,
                                        int* flag) {
  for (long long i = 0; i < max_polls; ++i) {
    if (bulk::try_wait(bar, parity)) return true;
    if (*abort_w) return false;
    if (i >= 8) __nanosleep(32);
  }
  if (!*abort_w) {
    *abort_w = 1;
    atomicExch(flag, 1);
  }
  return false;
}

// Warp-level: lane 0 waits, the warp learns the outcome, every lane acquires.
__device__ __forceinline__ bool ws_wait_warp(uint64_t* bar, uint32_t parity, long long max_polls,
                                             volatile int* abort_w, int* flag, int lane) {
  int ok = 1;
  if (lane == 0) ok = ws_wait(bar, parity, max_polls, abort_w, flag) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok && lane != 0) (void)bulk::try_wait(bar, parity);
  return ok != 0;
}

// Named barrier over `count` threads with an OR vote (true when any thread votes).
__device__ __forceinline__ bool ws_sync_or(int id, int count, bool vote) {
  uint32_t r;
  asm volatile(
      "{\n"
      ".reg .pred p, q;\n"
      "setp.ne.u32 p, %1, 0;\n"
      "bar.red.or.pred q, %2, %3, p;\n"
      "selp.u32 %0, 1, 0, q;\n"
      "}\n"
      : "=r"(r)
      : "r"((uint32_t)vote), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}

// Split one staged chunk into its terms (converter thread ct of 256).
// m stage: member m, half h (t 16 h ..): rows v of 16 t in the 128-byte
// swizzle (the 16-byte pair chunk c of row v at c ^ (v & 7)); W stage: box b
// (z 32 b ..): rows t of 32 z in the same swizzle.  TC t values per chunk.  Eight consecutive
// threads take eight consecutive volumes (A) or z (B).
template <int TC>
__device__ __forceinline__ void ws_convert(const WsPlan& P, const unsigned char* raw, unsigned char* set,
                                           const int (&mem)[4], const float* s_n, float inv_sw, int ct) {
  const int epc = P.epc, groups = TC / epc;
  unsigned char* a = set;
  unsigned char* b = set + P.nterm * P.a_term;
  for (int i = ct; i < 64 * groups; i += WS_CONV * 32) {
    const int v = i & 15, m = (i >> 4) & 3, gI = i >> 6;
    const int nre = ws_row(v, m, 0), nim = ws_row(v, m, 1);
    const uint32_t o_re = kchunk(NR, nre, gI * epc, epc), o_im = kchunk(NR, nim, gI * epc, epc);
    if (pick(mem, m) < 0) {
      for (int tI = 0; tI < P.nterm; ++tI) {
        *reinterpret_cast<uint4*>(a + tI * P.a_term + o_re) = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(a + tI * P.a_term + o_im) = make_uint4(0u, 0u, 0u, 0u);
      }
      continue;
    }
    const int t0 = gI * epc;  // epc t of one 16-t half
    const unsigned char* rowp = raw + ((TC / 16) * m + (t0 >> 4)) * WS_MBOX + v * 128;
    if (P.fp8) {
      const float sr = 1.f / s_n[nre], si = 1.f / s_n[nim];
      float vr[16], vi[16];
#pragma unroll
      for (int e = 0; e < 16; e += 2) {
        const int tt = (t0 & 15) + e;
        const float4 q = *reinterpret_cast<const float4*>(rowp + (((tt >> 1) ^ (v & 7)) << 4));
        vr[e] = q.x * sr;
        vi[e] = q.y * si;
        vr[e + 1] = q.z * sr;
        vi[e + 1] = q.w * si;
      }
      uint4 t0v, t1v, t2v;
      split16_e4m3(vr, t0v, t1v, t2v);
      *reinterpret_cast<uint4*>(a + o_re) = t0v;
      *reinterpret_cast<uint4*>(a + P.a_term + o_re) = t1v;
      *reinterpret_cast<uint4*>(a + 2 * P.a_term + o_re) = t2v;
      split16_e4m3(vi, t0v, t1v, t2v);
      *reinterpret_cast<uint4*>(a + o_im) = t0v;
      *reinterpret_cast<uint4*>(a + P.a_term + o_im) = t1v;
      *reinterpret_cast<uint4*>(a + 2 * P.a_term + o_im) = t2v;
    } else {
      float vr[8], vi[8];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        const int tt = (t0 & 15) + e;
        const float4 q = *reinterpret_cast<const float4*>(rowp + (((tt >> 1) ^ (v & 7)) << 4));
        vr[e] = q.x;
        vi[e] = q.y;
        vr[e + 1] = q.z;
        vi[e + 1] = q.w;
      }
      uint4 hi, lo;
      split8_bf16(vr, hi, lo);
      *reinterpret_cast<uint4*>(a + o_re) = hi;
      *reinterpret_cast<uint4*>(a + P.a_term + o_re) = lo;
      split8_bf16(vi, hi, lo);
      *reinterpret_cast<uint4*>(a + o_im) = hi;
      *reinterpret_cast<uint4*>(a + P.a_term + o_im) = lo;
    }
  }
  // B = W^T rows z < zn (z >= z4 reads the boxes' zero fill)
  const unsigned char* rw = raw + 4 * (TC / 16) * WS_MBOX;
  for (int i = ct; i < P.zn * groups; i += WS_CONV * 32) {
    const int z = i % P.zn, gI = i / P.zn;
    const unsigned char* box = rw + (z >> 5) * (32 * TC * 4) + (z & 3) * 4;
    const int zc = (z & 31) >> 2;
    const uint32_t o = kchunk(P.zn, z, gI * epc, epc);
    if (P.fp8) {
      float w[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int t = gI * 16 + e;
        w[e] = *reinterpret_cast<const float*>(box + t * 128 + ((zc ^ (t & 7)) << 4)) * inv_sw;
      }
      uint4 t0v, t1v, t2v;
      split16_e4m3(w, t0v, t1v, t2v);
      *reinterpret_cast<uint4*>(b + o) = t0v;
      *reinterpret_cast<uint4*>(b + P.b_term + o) = t1v;
      *reinterpret_cast<uint4*>(b + 2 * P.b_term + o) = t2v;
    } else {
      float w[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int t = gI * 8 + e;
        w[e] = *reinterpret_cast<const float*>(box + t * 128 + ((zc ^ (t & 7)) << 4));
      }
      uint4 hi, lo;
      split8_bf16(w, hi, lo);
      *reinterpret_cast<uint4*>(b + o) = hi;
      *reinterpret_cast<uint4*>(b + P.b_term + o) = lo;
    }
  }
}

template <int TC>
__global__ void __launch_bounds__(WS_THREADS, 1)
    k_batch_tikhonov_ws(const __grid_constant__ CUtensorMap mmap, const __grid_constant__ CUtensorMap wmap, WsPlan P,
                        const unsigned char* __restrict__ tabs, const float* __restrict__ class_scale,
                        const int* __restrict__ members, int nclass, const float2* __restrict__ m_hat, int ldm,
                        float2* __restrict__ x_hat, int ldx, int refine, int* flag, long long max_polls) {
  extern __shared__ float4 ws_smem4[];
  unsigned char* sm;
  {
    const uint32_t s = bulk::saddr(ws_smem4);
    sm = reinterpret_cast<unsigned char*>(ws_smem4) + (((s + 1023u) & ~1023u) - s);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nt = P.nt, nz = P.nz, zn = P.zn;
  const int NS = P.ns;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + P.off_bar);
  uint64_t* raw_full = bar + 0;     // [NS], one arrival + the copies' bytes
  uint64_t* raw_empty = bar + 4;    // [NS], one arrival per converter warp
  uint64_t* term_full = bar + 8;    // [NS], one arrival per converter warp
  uint64_t* term_empty = bar + 12;  // [NS], the MMAs that read the set (commit)
  uint64_t* acc_full = bar + 16;    // [2], the item's MMAs (commit)
  uint64_t* acc_empty = bar + 18;   // [2], one arrival per epilogue warp
  uint64_t* tab_full = bar + 20;    // the class tables' copy
  uint64_t* solve_bar = bar + 21;   // the solve MMAs (commit)
  uint64_t* drain_bar = bar + 22;   // every MMA issued (commit), before TMEM is freed
  uint64_t* sn_ready = bar + 23;    // [2] (FP8), one arrival per converter warp
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 25);
  volatile int* abort_w = reinterpret_cast<volatile int*>(bar + 26);
  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      bulk::bar_init(raw_full + i, 1);
      bulk::bar_init(raw_empty + i, WS_CONV);
      bulk::bar_init(term_full + i, WS_CONV);
      bulk::bar_init(term_empty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      bulk::bar_init(acc_full + i, 1);
      bulk::bar_init(acc_empty + i, WS_EPI);
      bulk::bar_init(sn_ready + i, WS_CONV);
    }
    bulk::bar_init(tab_full, 1);
    bulk::bar_init(solve_bar, 1);
    bulk::bar_init(drain_bar, 1);
    *abort_w = 0;
  }
  if (warp == 0) umma::tmem_alloc(tslot, 512);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t taddr = *tslot;
  const uint32_t sbase = bulk::saddr(sm);
  const int nchunks = (nt + TC - 1) / TC;
  const int nvc = P.nvc;
  const int acc_cols = P.nacc * zn, col_work = 2 * acc_cols;

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int gk = 0;  // chunks staged
      bool ok = true;
      for (int c = blockIdx.x; c < nclass && ok; c += gridDim.x) {
        int mem[4];
        for (int m = 0; m < 4; ++m) mem[m] = __ldg(members + 4 * c + m);
        int present = 0;
        for (int m = 0; m < 4; ++m) present += mem[m] >= 0;
        for (int vc = 0; vc < nvc && ok; ++vc)
          for (int kc = 0; kc < nchunks; ++kc, ++gk) {
            const int s = gk % NS;
            if (gk >= NS && !ws_wait(raw_empty + s, (uint32_t)((gk / NS) + 1) & 1u, max_polls, abort_w, flag)) {
              ok = false;
              break;
            }
            unsigned char* st = sm + P.off_raw + s * P.raw_stage;
            bulk::arrive_expect(raw_full + s, (unsigned)(present * (TC / 16) * WS_MBOX + P.nwb * 32 * TC * 4));
            for (int m = 0; m < 4; ++m)  // the chunk's 16-t halves: [half][volume][16 t]
              if (mem[m] >= 0)
                bulk::tensor_g2s_4d(st + (TC / 16) * m * WS_MBOX, &mmap, 0, vc * VB, kc * (TC / 16), mem[m],
                                    raw_full + s);
            for (int wb = 0; wb < P.nwb; ++wb)
              bulk::tensor_g2s_2d(st + 4 * (TC / 16) * WS_MBOX + wb * 32 * TC * 4, &wmap, 32 * wb, c * nt + kc * TC,
                                  raw_full + s);
          }
      }
      // no copy may still be landing when the CTA ends: the last load into each stage
      for (int s = 0; s < NS && s < gk; ++s)
        bulk::wait(raw_full + s, (uint32_t)((gk - 1 - s) / NS) & 1u, DRAIN_POLLS);
    }
  } else if (warp <= WS_CONV) {
    // ---------------- converters ----------------
    const int ct = threadIdx.x - 32;
    int gk = 0, it = 0;
    bool ok = true;
    for (int c = blockIdx.x; c < nclass && ok; c += gridDim.x) {
      int mem[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) mem[m] = __ldg(members + 4 * c + m);
      const float inv_sw = P.fp8 ? 1.f / __ldg(class_scale + c) : 1.f;
      for (int vc = 0; vc < nvc && ok; ++vc, ++it) {
        const int a = it & 1, v0 = vc * VB, nv = P.batch - v0 < VB ? P.batch - v0 : VB;
        float* s_n = reinterpret_cast<float*>(sm + P.off_sn) + a * NR;
        if (P.fp8) {
          // the epilogue is done with this scale buffer (item it - 2); then the
          // per-right-hand-side scales: the largest magnitude over t maps to 448
          if (it >= 2 &&
              !ws_wait_warp(acc_empty + a, (uint32_t)((it >> 1) + 1) & 1u, max_polls, abort_w, flag, lane)) {
            ok = false;
            break;
          }
          const int vm = ct >> 2, part = ct & 3, v = vm >> 2, m = vm & 3, f = pick(mem, m);
          float mr = 0.f, mi = 0.f;
          if (f >= 0 && v < nv) {
            const float2* src = m_hat + (size_t)f * ldm + (size_t)(v0 + v) * nt;
            for (int t = part; t < nt; t += 4) {
              const float2 x = __ldg(src + t);
              mr = fmaxf(mr, fabsf(x.x));
              mi = fmaxf(mi, fabsf(x.y));
            }
          }
          mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, 1));
          mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, 2));
          mi = fmaxf(mi, __shfl_xor_sync(0xffffffffu, mi, 1));
          mi = fmaxf(mi, __shfl_xor_sync(0xffffffffu, mi, 2));
          if (part == 0) {
            s_n[ws_row(v, m, 0)] = mr > 0.f ? mr / E4M3_MAX : 1.f;
            s_n[ws_row(v, m, 1)] = mi > 0.f ? mi / E4M3_MAX : 1.f;
          }
          __syncwarp();
          if (lane == 0) bulk::arrive(sn_ready + a);
          if (!ws_wait_warp(sn_ready + a, (uint32_t)(it >> 1) & 1u, max_polls, abort_w, flag, lane)) {
            ok = false;
            break;
          }
        }
        for (int kc = 0; kc < nchunks; ++kc, ++gk) {
          const int s = gk % NS;
          if (!ws_wait_warp(raw_full + s, (uint32_t)(gk / NS) & 1u, max_polls, abort_w, flag, lane) ||
              (gk >= NS &&
               !ws_wait_warp(term_empty + s, (uint32_t)((gk / NS) + 1) & 1u, max_polls, abort_w, flag, lane))) {
            ok = false;
            break;
          }
          ws_convert<TC>(P, sm + P.off_raw + s * P.raw_stage, sm + P.off_set + s * P.set_bytes, mem, s_n, inv_sw, ct);
          umma::fence_proxy_async();  // this lane's term writes, before the MMAs read them
          __syncwarp();
          if (lane == 0) {
            bulk::arrive(raw_empty + s);
            bulk::arrive(term_full + s);
          }
        }
      }
    }
  } else if (warp == WS_MMA_WARP) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc_main = P.fp8 ? idesc_e4m3(NR, zn) : idesc_bf16(NR, zn);
      int gk = 0, it = 0;
      bool ok = true;
      for (int c = blockIdx.x; c < nclass && ok; c += gridDim.x)
        for (int vc = 0; vc < nvc && ok; ++vc, ++it) {
          const int a = it & 1;
          if (it >= 2 && !ws_wait(acc_empty + a, (uint32_t)((it >> 1) + 1) & 1u, max_polls, abort_w, flag)) {
            ok = false;
            break;
          }
          umma::fence_after_sync();
          const uint32_t acc = taddr + (uint32_t)(a * acc_cols);
          for (int kc = 0; kc < nchunks; ++kc, ++gk) {
            const int s = gk % NS;
            if (!ws_wait(term_full + s, (uint32_t)(gk / NS) & 1u, max_polls, abort_w, flag)) {
              ok = false;
              break;
            }
            umma::fence_after_sync();
            const uint32_t a0 = sbase + P.off_set + s * P.set_bytes;
            const uint32_t b0 = a0 + P.nterm * P.a_term;
            const int ksteps = TC * P.esize / 32;  // K steps of 32 bytes per row
            for (int ks = 0; ks < ksteps; ++ks) {
              const uint32_t oa = ks * 2 * NR * 16, ob = ks * 2 * zn * 16;
              uint64_t A[3], B[3];
#pragma unroll
              for (int i = 0; i < 3; ++i) {
                A[i] = umma::desc(a0 + i * P.a_term + oa, NR * 16, 128);
                B[i] = umma::desc(b0 + i * P.b_term + ob, zn * 16, 128);
              }
              const uint32_t first = (kc > 0 || ks > 0) ? 1u : 0u;
              if (P.fp8) {
                mma_e4m3(acc, A[0], B[0], idesc_main, first);
                mma_e4m3(acc + zn, A[0], B[1], idesc_main, first);
                mma_e4m3(acc + zn, A[1], B[0], idesc_main, 1);
                mma_e4m3(acc + 2 * zn, A[0], B[2], idesc_main, first);
                mma_e4m3(acc + 2 * zn, A[1], B[1], idesc_main, 1);
                mma_e4m3(acc + 2 * zn, A[2], B[0], idesc_main, 1);
              } else {
                mma_bf16(acc, A[0], B[0], idesc_main, first);
                mma_bf16(acc + zn, A[0], B[1], idesc_main, first);
                mma_bf16(acc + zn, A[1], B[0], idesc_main, 1);
              }
            }
            umma::commit(term_empty + s);
          }
          if (ok) umma::commit(acc_full + a);
        }
      // every MMA this thread issued has finished before TMEM is freed
      umma::commit(drain_bar);
      bulk::wait(drain_bar, 0, DRAIN_POLLS);
    }
  } else {
    // ---------------- epilogue: solve and refinement ----------------
    const int et = threadIdx.x - WS_EPI0 * 32;
    const int n = 32 * (warp & 3) + lane;  // TMEM lane = right-hand side
    const uint32_t trow = taddr + ((uint32_t)(32 * (warp & 3)) << 16);
    const int v = n & 15, ri = (n >> 4) & 1, m = n >> 5;
    unsigned char* xh = sm + P.off_xh;
    unsigned char* xl = sm + P.off_xl;
    const uint32_t t_ch = sbase + P.off_tab, t_cl = t_ch + zn * zn * 4, t_gh = t_cl + zn * zn * 4,
                   t_gl = t_gh + zn * zn * 4;
    int tab_loads = 0;
    auto load_tables = [&](int c) {
      bulk::arrive_expect(tab_full, (unsigned)P.tab_bytes);
      bulk::g2s(sm + P.off_tab, tabs + (size_t)c * P.tab_bytes, (unsigned)P.tab_bytes, tab_full);
      ++tab_loads;
    };
    if (et == 0 && (int)blockIdx.x < nclass) load_tables(blockIdx.x);
    uint32_t sph = 0;  // solve barrier parity
    // the solve MMAs: one thread issues after every epilogue thread has written X
    auto solve = [&](uint32_t th, uint32_t tl) -> bool {
      umma::fence_proxy_async();
      umma::fence_before_sync();
      ws_sync_or(2, WS_EPI * 32, false);
      umma::fence_after_sync();
      if (et == 0) {
        issue_solve3(taddr + col_work, sbase + P.off_xh, sbase + P.off_xl, th, tl, zn);
        umma::commit(solve_bar);
      }
      const bool w_ok = ws_wait_warp(solve_bar, sph, max_polls, abort_w, flag, lane);
      sph ^= 1u;
      umma::fence_after_sync();
      return !ws_sync_or(2, WS_EPI * 32, !w_ok);
    };
    int it = 0, ci = 0;
    bool ok = true;
    for (int c = blockIdx.x; c < nclass && ok; c += gridDim.x, ++ci) {
      int mem[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) mem[q] = __ldg(members + 4 * c + q);
      const float sw = P.fp8 ? __ldg(class_scale + c) : 1.f;
      for (int vc = 0; vc < nvc && ok; ++vc, ++it) {
        const int a = it & 1, v0 = vc * VB, nv = P.batch - v0 < VB ? P.batch - v0 : VB;
        bool w_ok = ws_wait_warp(acc_full + a, (uint32_t)(it >> 1) & 1u, max_polls, abort_w, flag, lane);
        if (w_ok && vc == 0) w_ok = ws_wait_warp(tab_full, (uint32_t)ci & 1u, max_polls, abort_w, flag, lane);
        if (ws_sync_or(2, WS_EPI * 32, !w_ok)) {
          ok = false;
          break;
        }
        umma::fence_after_sync();
        const uint32_t acc = (uint32_t)(a * acc_cols);
        const float sn = P.fp8 ? reinterpret_cast<const float*>(sm + P.off_sn)[a * NR + n] * sw : 1.f;
        float x[4][16];
        // x0 = C b0
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (16 * j < zn) {
            float val[16];
            umma::tmem_ld16(trow + acc + 16 * j, val);
#pragma unroll
            for (int e = 0; e < 16; ++e) val[e] *= sn;
            put_x16(xh, xl, n, j, val);
          }
        }
        if (!solve(t_ch, t_cl)) {
          ok = false;
          break;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (16 * j < zn) umma::tmem_ld16(trow + col_work + 16 * j, x[j]);
        for (int r = 0; r < refine && ok; ++r) {
          // r = b - G' x
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (16 * j < zn) put_x16(xh, xl, n, j, x[j]);
          if (!solve(t_gh, t_gl)) {
            ok = false;
            break;
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (16 * j < zn) {
              float gx[16], d0[16], d1[16], d2[16];
              umma::tmem_ld16(trow + col_work + 16 * j, gx);
              umma::tmem_ld16(trow + acc + 16 * j, d0);
              umma::tmem_ld16(trow + acc + zn + 16 * j, d1);
              if (P.fp8) umma::tmem_ld16(trow + acc + 2 * zn + 16 * j, d2);
              float rr[16];
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const float bb = P.fp8 ? sn * (d0[e] + 0.0625f * d1[e] + 0.00390625f * d2[e]) : d0[e] + d1[e];
                rr[e] = bb - gx[e];
              }
              put_x16(xh, xl, n, j, rr);
            }
          }
          // x += C r
          if (!solve(t_ch, t_cl)) {
            ok = false;
            break;
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (16 * j < zn) {
              float cr[16];
              umma::tmem_ld16(trow + col_work + 16 * j, cr);
#pragma unroll
              for (int e = 0; e < 16; ++e) x[j][e] += cr[e];
            }
          }
        }
        if (!ok) break;
        // the accumulators are read: the MMAs of item it + 2 may overwrite them
        umma::fence_before_sync();
        __syncwarp();
        if (lane == 0) bulk::arrive(acc_empty + a);
        // x_hat[f][v * nz + z]: lanes 0-15 hold the real parts, lanes 16-31 the imaginary ones
        {
          const int fm = pick(mem, m);
          const bool writer = ri == 0 && v < nv && fm >= 0;
          float2* dst = x_hat + (size_t)(fm >= 0 ? fm : 0) * ldx + (size_t)(v0 + (v < nv ? v : 0)) * nz;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (16 * j < zn) {
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const float im = __shfl_down_sync(0xffffffffu, x[j][e], 16);
                const int z = 16 * j + e;
                if (writer && z < nz) dst[z] = make_float2(x[j][e], im);
              }
            }
          }
        }
      }
      // every solve MMA of this class has completed: the tables may be replaced
      if (ok && et == 0 && c + (int)gridDim.x < nclass) load_tables(c + gridDim.x);
    }
    if (et == 0 && tab_loads) bulk::wait(tab_full, (uint32_t)(tab_loads - 1) & 1u, DRAIN_POLLS);
  }
  __syncwarp();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (warp == 0) umma::tmem_dealloc(taddr, 512);
}

// Per-class FP8 scale of W_hat: max |W| / 448.
__global__ void k_class_absmax(const float* __restrict__ what, int per_class, int nclass, float* __restrict__ out) {
  __shared__ float red[32];
  for (int c = blockIdx.x; c < nclass; c += gridDim.x) {
    float m = 0.f;
    const float* w = what + (size_t)c * per_class;
    for (int i = threadIdx.x; i < per_class; i += blockDim.x) m = fmaxf(m, fabsf(w[i]));
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
      m = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
      for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (threadIdx.x == 0) out[c] = m > 0.f ? m / E4M3_MAX : 1.f;
    }
    __syncthreads();
  }
}

// C = (G + lambda I)^-1 (FP64 Cholesky -> FP32) and G + lambda I (FP32), rows padded to z4.
__global__ void __launch_bounds__(128) k_factor_tik(const double* __restrict__ gram, int nz, double lambda,
                                                    float* __restrict__ cinv, float* __restrict__ glam) {
  extern __shared__ double smd[];
  const int ld = nz + 1;
  double* s_a = smd;
  double* s_l = smd + nz * ld;
  const int c = blockIdx.x;
  const int z4 = (nz + 3) & ~3;
  const double* g = gram + (size_t)c * nz * nz;
  for (int idx = threadIdx.x; idx < nz * nz; idx += blockDim.x) {
    const int i = idx / nz, j = idx - i * nz;
    const double v = g[idx] + (i == j ? lambda : 0.0);
    s_a[i * ld + j] = v;
    glam[((size_t)c * nz + i) * z4 + j] = (float)v;
  }
  for (int idx = threadIdx.x; idx < nz * (z4 - nz); idx += blockDim.x) {
    const int i = idx / (z4 - nz), j = nz + idx % (z4 - nz);
    glam[((size_t)c * nz + i) * z4 + j] = 0.f;
  }
  __syncthreads();
  for (int j = 0; j < nz; ++j) {
    if (threadIdx.x == 0) s_a[j * ld + j] = sqrt(s_a[j * ld + j]);
    __syncthreads();
    const double d = s_a[j * ld + j];
    for (int i = j + 1 + threadIdx.x; i < nz; i += blockDim.x) s_a[i * ld + j] /= d;
    __syncthreads();
    const int rem = nz - j - 1;
    for (int idx = threadIdx.x; idx < rem * rem; idx += blockDim.x) {
      const int i = j + 1 + idx / rem, l = j + 1 + idx % rem;
      if (l <= i) s_a[i * ld + l] -= s_a[i * ld + j] * s_a[l * ld + j];
    }
    __syncthreads();
  }
  for (int col = threadIdx.x; col < nz; col += blockDim.x) {
    for (int i = 0; i < col; ++i) s_l[i * ld + col] = 0.0;
    for (int i = col; i < nz; ++i) {
      double acc = (i == col) ? 1.0 : 0.0;
      for (int kk = col; kk < i; ++kk) acc -= s_a[i * ld + kk] * s_l[kk * ld + col];
      s_l[i * ld + col] = acc / s_a[i * ld + i];
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nz * z4; idx += blockDim.x) {
    const int i = idx / z4, j = idx - i * z4;
    double acc = 0.0;
    if (j < nz)
      for (int kk = (i > j ? i : j); kk < nz; ++kk) acc += s_l[kk * ld + i] * s_l[kk * ld + j];
    cinv[((size_t)c * nz + i) * z4 + j] = (float)acc;
  }
}

// Solve tables per class: C and G + lambda I as TF32 hi / lo in the canonical
// K-major layout of a B operand with zn rows (z) and K = w (both symmetric).
__global__ void k_solve_tables(const float* __restrict__ cinv, const float* __restrict__ glam, int nz, int z4, int zn,
                               int nclass, unsigned char* __restrict__ tabs) {
  const int per = zn * zn;
  const size_t total = (size_t)nclass * per;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t c = i / per;
    const int rem = (int)(i - c * per), z = rem / zn, w = rem - z * zn;
    float vc = 0.f, vg = 0.f;
    if (z < nz && w < nz) {
      vc = cinv[(c * nz + z) * z4 + w];
      vg = glam[(c * nz + z) * z4 + w];
    }
    float ch, cl, gh, gl;
    umma::split_tf32(vc, ch, cl);
    umma::split_tf32(vg, gh, gl);
    const size_t o = (size_t)(((w >> 2) * zn + z) * 16 + (w & 3) * 4);
    unsigned char* t = tabs + c * (size_t)(4 * per * 4);
    *reinterpret_cast<float*>(t + o) = ch;
    *reinterpret_cast<float*>(t + per * 4 + o) = cl;
    *reinterpret_cast<float*>(t + 2 * per * 4 + o) = gh;
    *reinterpret_cast<float*>(t + 3 * per * 4 + o) = gl;
  }
}

}  // namespace

size_t batch_tikhonov_smem_bytes(int nt, int nz) {
  const BtPlan a = make_plan(nt, nz, 0, 1), b = make_plan(nt, nz, 1, 1);
  return (size_t)(a.total > b.total ? a.total : b.total);
}

// Build (once per handle) the per-class FP8 scales and (per lambda) C, G + lambda I
// and their BF16 solve tables.
ctof_status batch_tikhonov_prepare(ctof_kernel_s* k, double lambda, cudaStream_t st) {
  const int zn = rup(k->nz, 16);
  if (!k->d_bt_cinv) {
    // one allocation, each part starting on a 256-byte boundary (the tables are
    // read with 16-byte asynchronous copies)
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t fl = al((size_t)k->nclass * k->nz * k->z4 * sizeof(float));
    const size_t sw = al((size_t)k->nclass * sizeof(float));
    const size_t tab = (size_t)k->nclass * 4 * zn * zn * 4;
    void* p = nullptr;
    if (cudaMalloc(&p, 2 * fl + sw + tab) != cudaSuccess) {
      cudaGetLastError();
      return CTOF_ENOMEM;
    }
    unsigned char* b = static_cast<unsigned char*>(p);
    k->d_bt_cinv = reinterpret_cast<float*>(b);
    k->d_bt_glam = reinterpret_cast<float*>(b + fl);
    k->d_bt_sw = reinterpret_cast<float*>(b + 2 * fl);
    k->d_bt_tab = b + 2 * fl + sw;
    k->bt_lambda = -1.0;
    k_class_absmax<<<152 * 4, 256, 0, st>>>(k->d_what, k->nt * k->z4, k->nclass, k->d_bt_sw);
    CTOF_CUDA_TRY(cudaGetLastError());
  }
  if (k->bt_lambda != lambda) {
    const size_t fsm = (size_t)2 * k->nz * (k->nz + 1) * sizeof(double);
    CTOF_CUDA_TRY(cudaFuncSetAttribute(k_factor_tik, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm));
    k_factor_tik<<<k->nclass, 128, fsm, st>>>(k->d_gram, k->nz, lambda, k->d_bt_cinv, k->d_bt_glam);
    CTOF_CUDA_TRY(cudaGetLastError());
    k_solve_tables<<<152 * 8, 256, 0, st>>>(k->d_bt_cinv, k->d_bt_glam, k->nz, k->z4, zn, k->nclass, k->d_bt_tab);
    CTOF_CUDA_TRY(cudaGetLastError());
    k->bt_lambda = lambda;
  }
  return CTOF_OK;
}

ctof_status batch_tikhonov_contract(const ctof_kernel_s* k, int precision, int batch, const float2* m_hat, int ldm,
                                    float2* x_hat, int ldx, int refine, cudaStream_t st) {
  const int fp8 = precision == CTOF_FP8E4M3 ? 1 : 0;
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, k->device);
  const int grid = k->nclass < nsm ? k->nclass : nsm;
  if (k->nt % 16 == 0 && rup(k->nz, 16) <= 64) {
    // warp-specialised kernel: m_hat [f][v][t] and W_hat [c t][z] staged by tensor maps
    const WsPlan W = make_ws_plan(k->nt, k->nz, fp8, batch);
    if (W.total <= 227 * 1024) {
      // m_hat element (t = 16 h + tt, v, f) as a 4-D tensor (tt, v, h, f): one box
      // of 16 tt x 16 volumes x TC/16 halves per member lands as [half][volume][16 t]
      CUtensorMap mmap, wmap;
      const unsigned long long mdims[4] = {16, (unsigned long long)batch, (unsigned long long)k->nt / 16,
                                           (unsigned long long)k->nf};
      const unsigned long long mstr[3] = {(unsigned long long)k->nt * 8, 16 * 8, (unsigned long long)ldm * 8};
      const unsigned mbox[4] = {16, VB, (unsigned)W.tc / 16, 1};
      const unsigned long long wdims[2] = {(unsigned long long)k->z4, (unsigned long long)k->nt * k->nclass};
      const unsigned long long wstr[1] = {(unsigned long long)k->z4 * 4};
      const unsigned wbox[2] = {32, (unsigned)W.tc};
      if (ctof_encode_map(&mmap, 8, 4, m_hat, mdims, mstr, mbox, 128) == CTOF_OK &&
          ctof_encode_map(&wmap, 4, 2, k->d_what, wdims, wstr, wbox, 128) == CTOF_OK) {
        auto kern = k_batch_tikhonov_ws<32>;
        CTOF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, W.total));
        kern<<<grid, WS_THREADS, W.total, st>>>(mmap, wmap, W, k->d_bt_tab, k->d_bt_sw, k->d_members, k->nclass,
                                                m_hat, ldm, x_hat, ldx, refine, k->d_flags, k->max_polls);
        CTOF_CUDA_TRY(cudaGetLastError());
        return CTOF_OK;
      }
      ctof_set_last_error_text("");  // a buffer the maps cannot take: the kernel below stages by plain copies
    }
  }
  const BtPlan P = make_plan(k->nt, k->nz, fp8, batch);
  if (P.total > 227 * 1024) return CTOF_EUNSUPPORTED;
  CTOF_CUDA_TRY(cudaFuncSetAttribute(k_batch_tikhonov_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, P.total));
  k_batch_tikhonov_tc<<<grid, BT_THREADS, P.total, st>>>(P, k->d_what, k->d_bt_tab, k->d_bt_sw, k->d_members,
                                                          k->nclass, m_hat, ldm, x_hat, ldx, refine, k->d_flags,
                                                          k->max_polls);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}
