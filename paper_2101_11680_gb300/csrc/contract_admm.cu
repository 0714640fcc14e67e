// Fused ADMM x-update per frequency class (Eq. 11 in the lateral Fourier
// domain, one iteration of the normal-equation solve):
//   b     = W_hat^T c_hat / s + s_hat - L x_hat_prev          (Z x 8 real)
//   x_hat = x_hat_prev + H^-1 b
//   Kx    = W_hat x_hat / s                                     (T x 8 real)
// with L = (|dx|^2 + |dy|^2 + 1) I + Dz^T Dz and H = W_hat^T W_hat / s^2 + L,
// i.e. x_hat = H^-1 (W_hat^T (K x_hat_prev + c_hat)/s + s_hat).  The 8 real
// right-hand sides are the real/imaginary parts of the up-to-4 frequencies
// of one class (they share the real matrix W_hat).  W_hat is streamed once
// per iteration; every contraction runs on the warp-level tensor-core MMA
// (m16n8k8, TF32 inputs, FP32 accumulation) with each operand split into a
// TF32 high part and a TF32 remainder (three MMAs per tile: lo*hi + hi*lo +
// hi*hi), which keeps FP32-level accuracy; N = 8 is exactly the 8 real
// right-hand sides of a class.
//
// Two kernels:
//
// k_contract_admm_pipe (used whenever two or more stages fit in shared
// memory; 128 x 128 x 48 x 256 takes three): one CTA per SM, a producer warp
// and eight consumer warps.  The producer streams each class into a ring of
// shared-memory stages with bulk asynchronous copies (cp.async.bulk, one per
// contiguous block: the class's W_hat and H^-1 blocks and each member's
// c_hat, s_hat and x_hat rows, 14 requests of up to 48 KB for a class of four
// members), completing on the stage's mbarrier; consumers release a stage
// through a second mbarrier once its class is done.  W_hat and H^-1 are read
// from ADMM copies laid out in 8 x 8 blocks whose 64 words are permuted so
// that both the forward fragments (row <-> lane group, column <-> lane in
// group) and the adjoint's transposed fragments load without shared-memory
// bank conflicts from the flat bulk copy:
//   word(i, j) = 32 (j / 4) + 4 ((i + 4 (j / 4)) mod 8) + j mod 4,
//   i = row mod 8, j = column mod 8.
// Per class the consumers run four phases between named barriers:
//   A  adjoint partial sums, the eight warps splitting the t (K) steps;
//   B  b = sum of the partials / s + s_hat - L x_prev, split for the MMA;
//   C  x_new = x_prev + H^-1 b (one warp per 16-row z tile), stored;
//   D  Kx = W x_new / s (warps over 16-row t tiles), stored.
// Every wait is bounded: a wait that runs out sets the handle's sticky flag
// and the CTA stops (the consumers vote at their next barrier, the producer
// stops issuing and waits, with a fixed drain limit, for the copies it has
// in flight).
//
// k_contract_admm (fallback for class blocks too large for two stages):
// persistent CTAs of 8 warps walk the classes, two per SM where their shared
// memory fits (one buffer each), otherwise one CTA per SM prefetching class
// i+1 with 16-byte cp.async copies into a second buffer; shared W_hat rows
// are padded to a stride zp with zp/4 odd so that the MMA fragment loads hit
// distinct banks.
//   adjoint part: warps split the t (K) steps over all z tiles; partial
//                 results meet in shared memory.
//   H^-1 part:    FP32 FMA, thread per (z, member).
//   forward part: one warp per 16-row tile of t.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ctof_internal.h"

namespace {

constexpr int AD_THREADS = 256;
constexpr int AD_WARPS = AD_THREADS / 32;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Rows x chunks (16-byte) copy with per-thread incremental (row, chunk) walk:
// element i = tid + k*AD_THREADS, row = i / cpr, chunk = i % cpr, without divisions
// in the loop.
__device__ __forceinline__ void copy_rows(float* dst, int dst_stride, const float* src, int src_stride, int rows,
                                          int cpr) {
  const int tid = threadIdx.x;
  int r = tid / cpr, q = tid - r * cpr;
  const int dr = AD_THREADS / cpr, dq = AD_THREADS - dr * cpr;
  while (r < rows) {
    cp_async16(dst + r * dst_stride + 4 * q, src + (size_t)r * src_stride + 4 * q);
    r += dr;
    q += dq;
    if (q >= cpr) {
      q -= cpr;
      ++r;
    }
  }
}

struct AdmmLayout {
  int nt, nz, z4, zp, zm, tm, ntp;
  int nbuf;
  int buf_floats;                         // floats per buffer
  int off_w, off_h, off_c, off_s, off_x;  // within a buffer
  int off_ch, off_cl, off_xh, off_xl;     // split B operands [tm][8] / [zm][8]
  int off_part, off_b;                    // after the buffers
  int total_floats;
};

// 3xTF32 split: x = hi + lo with hi, lo representable in TF32.
__device__ __forceinline__ void split_tf32(float x, unsigned& hi, unsigned& lo) {
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(hi) : "f"(x));
  const float r = x - __uint_as_float(hi);
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(lo) : "f"(r));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// d += A B in 3xTF32 (A_lo B_hi + A_hi B_lo + A_hi B_hi, small terms first), A
// given in FP32 and split here, B already split.
__device__ __forceinline__ void mma_3xtf32(float (&d)[4], const float (&a)[4], unsigned bh0, unsigned bh1,
                                           unsigned bl0, unsigned bl1) {
  unsigned ah[4], al[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) split_tf32(a[i], ah[i], al[i]);
  mma_tf32(d, al, bh0, bh1);
  mma_tf32(d, ah, bl0, bl1);
  mma_tf32(d, ah, bh0, bh1);
}

// All threads issue the 16-byte asynchronous copies of class c into `buf`
// (W_hat and H^-1 rows into padded shared rows, member vectors contiguously).
__device__ __forceinline__ void issue_class(const AdmmLayout& L, float* buf, int c, const int* __restrict__ members,
                                            const float* __restrict__ what, const float* __restrict__ hinv,
                                            const float2* __restrict__ c_hat, int ldt,
                                            const float2* __restrict__ s_hat, const float2* __restrict__ x_hat,
                                            int ldz) {
  const int q4 = L.z4 >> 2;
  copy_rows(buf + L.off_w, L.zp, what + (size_t)c * L.nt * L.z4, L.z4, L.nt, q4);
  copy_rows(buf + L.off_h, L.zp, hinv + (size_t)c * L.nz * L.z4, L.z4, L.nz, q4);
  const int tid = threadIdx.x;
  const int cper = L.ntp >> 1, zper = L.z4 >> 1;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int f = members[c * 4 + m];
    if (f < 0) continue;  // absent member: its smem slot keeps stale finite data, never stored
    for (int j = tid; j < cper; j += AD_THREADS)
      cp_async16(buf + L.off_c + (m * L.ntp + 2 * j) * 2, c_hat + (size_t)f * ldt + 2 * j);
    for (int j = tid; j < zper; j += AD_THREADS) {
      cp_async16(buf + L.off_s + (m * L.z4 + 2 * j) * 2, s_hat + (size_t)f * ldz + 2 * j);
      cp_async16(buf + L.off_x + (m * L.z4 + 2 * j) * 2, x_hat + (size_t)f * ldz + 2 * j);
    }
  }
}

__global__ void __launch_bounds__(AD_THREADS, 2) k_contract_admm(
    AdmmLayout L, const float* __restrict__ what, const float* __restrict__ hinv, const float* __restrict__ lap,
    const int* __restrict__ members, int nclass, const float2* __restrict__ c_hat, int ldt,
    const float2* __restrict__ s_hat, float2* __restrict__ x_hat, int ldz, float2* __restrict__ kx_hat,
    float inv_s) {
  extern __shared__ __align__(16) float sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, tg = lane & 3;  // MMA fragment coordinates
  const int nt = L.nt, nz = L.nz, zp = L.zp;
  float* s_part = sm + L.off_part;                               // [AD_WARPS][zm][8], aliases s_ch/s_cl
  float* s_b = sm + L.off_b;                                     // [zm][8]
  unsigned* s_ch = reinterpret_cast<unsigned*>(sm + L.off_ch);   // [tm][8] c_hat hi (TF32 bits)
  unsigned* s_cl = reinterpret_cast<unsigned*>(sm + L.off_cl);   // [tm][8] c_hat lo
  unsigned* s_xh = reinterpret_cast<unsigned*>(sm + L.off_xh);   // [zm][8] x_new hi
  unsigned* s_xl = reinterpret_cast<unsigned*>(sm + L.off_xl);   // [zm][8] x_new lo
  // zero all shared memory once (padding rows/columns are never written by the copies)
  for (int i = tid; i < L.total_floats; i += AD_THREADS) sm[i] = 0.f;
  __syncthreads();
  int c = blockIdx.x;
  if (c >= nclass) return;
  issue_class(L, sm, c, members, what, hinv, c_hat, ldt, s_hat, x_hat, ldz);
  cp_async_commit();
  const int ksteps_t = L.tm >> 3;  // K steps over t (adjoint)
  const int mtiles_z = L.zm >> 4;  // M tiles over z (adjoint)
  const int ksteps_z = (nz + 7) >> 3;
  const int mtiles_t = L.tm >> 4;
  for (int it = 0; c < nclass; ++it, c += gridDim.x) {
    const int cn = c + gridDim.x;
    const int bi = L.nbuf == 2 ? (it & 1) : 0;
    float* buf = sm + bi * L.buf_floats;
    if (L.nbuf == 2) {
      if (cn < nclass)
        issue_class(L, sm + (bi ^ 1) * L.buf_floats, cn, members, what, hinv, c_hat, ldt, s_hat, x_hat, ldz);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    int mem[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) mem[m] = members[c * 4 + m];
    const float* s_w = buf + L.off_w;
    const float* s_h = buf + L.off_h;
    const float2* s_c = reinterpret_cast<const float2*>(buf + L.off_c);  // [4][ntp]
    const float2* s_s = reinterpret_cast<const float2*>(buf + L.off_s);  // [4][z4]
    const float2* s_x = reinterpret_cast<const float2*>(buf + L.off_x);  // [4][z4]

    // ---- split c_hat into TF32 hi/lo, laid out [t][r] (r = 2 member + component) ----
    for (int i = tid; i < nt * 4; i += AD_THREADS) {
      const int t = i >> 2, m = i & 3;
      const float2 v = s_c[m * L.ntp + t];
      unsigned h0, l0, h1, l1;
      split_tf32(v.x, h0, l0);
      split_tf32(v.y, h1, l1);
      *reinterpret_cast<uint2*>(s_ch + t * 8 + 2 * m) = make_uint2(h0, h1);
      *reinterpret_cast<uint2*>(s_cl + t * 8 + 2 * m) = make_uint2(l0, l1);
    }
    __syncthreads();
    // ---- adjoint: D[z][r] = sum_t W[t][z] c[t][r]; warps split the t (K) steps ----
    {
      float acc[4][4];
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[mt][i] = 0.f;
      for (int ks = warp; ks < ksteps_t; ks += AD_WARPS) {
        const int ta = ks * 8 + tg, tb = ta + 4;
        const unsigned bh0 = s_ch[ta * 8 + g], bh1 = s_ch[tb * 8 + g];
        const unsigned bl0 = s_cl[ta * 8 + g], bl1 = s_cl[tb * 8 + g];
        const float* wa = s_w + ta * zp + g;
        const float* wb = s_w + tb * zp + g;
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
          if (mt < mtiles_z) {
            const float a[4] = {wa[mt * 16], wa[mt * 16 + 8], wb[mt * 16], wb[mt * 16 + 8]};
            mma_3xtf32(acc[mt], a, bh0, bh1, bl0, bl1);
          }
        }
      }
      __syncthreads();  // the partial sums overwrite the split c_hat operands
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        if (mt < mtiles_z) {
          float* p = s_part + (warp * L.zm + mt * 16 + g) * 8 + 2 * tg;
          *reinterpret_cast<float2*>(p) = make_float2(acc[mt][0], acc[mt][1]);
          *reinterpret_cast<float2*>(p + 64) = make_float2(acc[mt][2], acc[mt][3]);
        }
      }
    }
    __syncthreads();
    // ---- b = W^T c / s + s_hat - L x_prev ----
    {
      const float dl = lap[c] + 1.0f;
      const int nw = ksteps_t < AD_WARPS ? ksteps_t : AD_WARPS;
      for (int i = tid; i < nz * 8; i += AD_THREADS) {
        const int z = i >> 3, r = i & 7, m = r >> 1;
        float a = 0.f;
        for (int w = 0; w < nw; ++w) a += s_part[w * L.zm * 8 + i];
        const float* xm = reinterpret_cast<const float*>(s_x + m * L.z4);
        const int cpn = r & 1;
        const float xz = xm[2 * z + cpn];
        float lx = dl * xz;
        if (z > 0) lx += xz - xm[2 * (z - 1) + cpn];
        if (z < nz - 1) lx -= xm[2 * (z + 1) + cpn] - xz;
        const float sv = reinterpret_cast<const float*>(s_s + m * L.z4)[2 * z + cpn];
        s_b[i] = a * inv_s + sv - lx;
      }
    }
    __syncthreads();
    // ---- x_new = x_prev + H^-1 b; x_new stored split for the forward MMA ----
    for (int i = tid; i < nz * 4; i += AD_THREADS) {
      const int z = i >> 2, m = i & 3;
      float2 acc = s_x[m * L.z4 + z];
      const float* hr = s_h + z * zp;
      for (int w = 0; w < L.z4; w += 4) {
        const float4 h = *reinterpret_cast<const float4*>(hr + w);
        const float2 b0 = *reinterpret_cast<const float2*>(s_b + (w + 0) * 8 + 2 * m);
        const float2 b1 = *reinterpret_cast<const float2*>(s_b + (w + 1) * 8 + 2 * m);
        const float2 b2 = *reinterpret_cast<const float2*>(s_b + (w + 2) * 8 + 2 * m);
        const float2 b3 = *reinterpret_cast<const float2*>(s_b + (w + 3) * 8 + 2 * m);
        acc.x += h.x * b0.x + h.y * b1.x + h.z * b2.x + h.w * b3.x;
        acc.y += h.x * b0.y + h.y * b1.y + h.z * b2.y + h.w * b3.y;
      }
      unsigned h0, l0, h1, l1;
      split_tf32(acc.x, h0, l0);
      split_tf32(acc.y, h1, l1);
      *reinterpret_cast<uint2*>(s_xh + z * 8 + 2 * m) = make_uint2(h0, h1);
      *reinterpret_cast<uint2*>(s_xl + z * 8 + 2 * m) = make_uint2(l0, l1);
      if (mem[m] >= 0) x_hat[(size_t)mem[m] * ldz + z] = acc;
    }
    __syncthreads();
    // ---- forward: Kx[t][r] = sum_z W[t][z] x_new[z][r] / s; warp per 16-row t tile ----
    for (int mt = warp; mt < mtiles_t; mt += AD_WARPS) {
      const int t0 = mt * 16;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      const float* w0 = s_w + (t0 + g) * zp + tg;
      const float* w1 = w0 + 8 * zp;
      for (int ks = 0; ks < ksteps_z; ++ks) {
        const int k0 = ks * 8;
        const float a[4] = {w0[k0], w1[k0], w0[k0 + 4], w1[k0 + 4]};
        const int bi0 = (k0 + tg) * 8 + g, bi1 = bi0 + 32;
        mma_3xtf32(acc, a, s_xh[bi0], s_xh[bi1], s_xl[bi0], s_xl[bi1]);
      }
      // lane (g, tg) holds r = 2 tg, 2 tg + 1 (member tg) at t0 + g and t0 + g + 8
      if (mem[tg] >= 0) {
        float2* dst = kx_hat + (size_t)mem[tg] * ldt;
        if (t0 + g < nt) dst[t0 + g] = make_float2(acc[0] * inv_s, acc[1] * inv_s);
        if (t0 + g + 8 < nt) dst[t0 + g + 8] = make_float2(acc[2] * inv_s, acc[3] * inv_s);
      }
    }
    __syncthreads();
    if (L.nbuf == 1 && cn < nclass) {
      issue_class(L, sm, cn, members, what, hinv, c_hat, ldt, s_hat, x_hat, ldz);
      cp_async_commit();
    }
  }
}



AdmmLayout make_layout(int nt, int nz, int nbuf) {
  AdmmLayout L;
  L.nt = nt;
  L.nz = nz;
  L.z4 = (nz + 3) & ~3;
  L.zm = (nz + 15) & ~15;
  L.zp = ((L.zm >> 2) & 1) ? L.zm : L.zm + 4;
  L.tm = (nt + 15) & ~15;
  L.ntp = (nt + 1) & ~1;
  L.nbuf = nbuf;
  L.off_w = 0;
  L.off_h = L.off_w + L.tm * L.zp;
  L.off_c = L.off_h + L.nz * L.zp;
  L.off_s = L.off_c + ((4 * L.ntp * 2 + 3) & ~3);
  L.off_x = L.off_s + 4 * L.z4 * 2;
  L.buf_floats = L.off_x + 4 * L.z4 * 2;
  // the adjoint's split c_hat operands and its per-warp partial sums share one region
  L.off_ch = nbuf * L.buf_floats;
  L.off_cl = L.off_ch + L.tm * 8;
  L.off_part = L.off_ch;
  const int shared_region = L.tm * 16 > AD_WARPS * L.zm * 8 ? L.tm * 16 : AD_WARPS * L.zm * 8;
  L.off_xh = L.off_ch + shared_region;
  L.off_xl = L.off_xh + L.zm * 8;
  L.off_b = L.off_xl + L.zm * 8;
  L.total_floats = L.off_b + L.zm * 8;
  return L;
}


// ======================= pipelined kernel (bulk-copy stage ring) =======================

constexpr int PIPE_CONS_WARPS = 8;
constexpr int PIPE_CONS_THREADS = 32 * PIPE_CONS_WARPS;
constexpr int PIPE_THREADS = PIPE_CONS_THREADS + 32;  // + one producer warp
constexpr long long PIPE_DRAIN_POLLS = 1ll << 24;     // polls of the waits that follow a timeout
constexpr int PIPE_SMEM_LIMIT = 227 * 1024;

inline int rup(int x, int m) { return (x + m - 1) / m * m; }

struct PipePlan {
  int nt, nz, z4, zm, tm, ntp;
  int cs, sz;                     // words per member row: c stage (2 tm + 8), s / x stages (2 z4 + 8)
  int stages;
  int o_w, o_h, o_c, o_s, o_x, o_hdr;  // byte offsets within a stage
  int stage_bytes;
  int o_part, o_bh, o_bl, o_xh, o_xl, o_bar;  // byte offsets after the stages
  int total;
  unsigned w_bytes, h_bytes, c_bytes, v_bytes;  // bulk copy sizes
};

PipePlan make_pipe_plan(int nt, int nz, int stages) {
  PipePlan P{};
  P.nt = nt;
  P.nz = nz;
  P.z4 = rup(nz, 4);
  P.zm = rup(nz, 16);
  P.tm = rup(nt, 16);
  P.ntp = rup(nt, 2);
  P.cs = 2 * P.tm + 8;  // = 8 mod 32 words: the adjoint's B fragments are conflict-free
  P.sz = 2 * P.z4 + 8;  // member rows 8 banks apart
  P.stages = stages;
  P.o_w = 0;
  P.o_h = P.o_w + P.tm * P.zm * 4;
  P.o_c = P.o_h + P.zm * P.zm * 4;
  P.o_s = P.o_c + 4 * P.cs * 4;
  P.o_x = P.o_s + 4 * P.sz * 4;
  P.o_hdr = P.o_x + 4 * P.sz * 4;  // 4 member indices + the diagonal of L (written by the producer)
  P.stage_bytes = rup(P.o_hdr + 32, 128);
  P.o_part = stages * P.stage_bytes;
  P.o_bh = P.o_part + PIPE_CONS_WARPS * P.zm * 8 * 4;
  P.o_bl = P.o_bh + P.zm * 8 * 4;
  P.o_xh = P.o_bl + P.zm * 8 * 4;
  P.o_xl = P.o_xh + P.zm * 8 * 4;
  P.o_bar = P.o_xl + P.zm * 8 * 4;
  P.total = P.o_bar + 2 * stages * 8 + 16;  // full[S], empty[S], abort word
  P.w_bytes = (unsigned)(P.tm * P.zm * 4);
  P.h_bytes = (unsigned)(P.zm * P.zm * 4);
  P.c_bytes = (unsigned)(P.ntp * 8);
  P.v_bytes = (unsigned)(P.z4 * 8);
  return P;
}

// Most stages (up to 4) that fit, or 0 when fewer than two do.
int pipe_stages(int nt, int nz) {
  if (nz > 64) return 0;
  for (int s = 4; s >= 2; --s)
    if (make_pipe_plan(nt, nz, s).total <= PIPE_SMEM_LIMIT) return s;
  return 0;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait for the phase of the given parity (false: gave up).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long max_polls) {
  for (long long i = 0; i < max_polls; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// Bulk global -> shared copy completing `bytes` of transaction count on `bar`
// (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Barrier 1 over the 256 consumer threads (the producer warp never joins it).
__device__ __forceinline__ void cons_sync() { asm volatile("bar.sync 1, 256;\n" ::: "memory"); }
__device__ __forceinline__ int cons_sync_or(int v) {
  int out;
  asm volatile(
      "{\n"
      ".reg .pred q, p;\n"
      "setp.ne.s32 q, %1, 0;\n"
      "bar.red.or.pred p, 1, 256, q;\n"
      "selp.s32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(out)
      : "r"(v)
      : "memory");
  return out;
}

// W_hat -> [class][tm/8][zm/8][64] and H^-1 -> [class][zm/8][zm/8][64] in the
// permuted 8 x 8 block layout described at the top of this file (zero padding).
__global__ void k_admm_reorder(const float* __restrict__ src, int rows, int cols, int ld, int rm, int cm,
                               float* __restrict__ dst, int nclass) {
  const size_t per = (size_t)rm * cm, total = per * nclass;
  const int cb_n = cm >> 3;
  for (size_t d = (size_t)blockIdx.x * blockDim.x + threadIdx.x; d < total; d += (size_t)gridDim.x * blockDim.x) {
    const size_t c = d / per;
    const int rem = (int)(d - c * per), blk = rem >> 6, w = rem & 63;
    const int rb = blk / cb_n, cb = blk - rb * cb_n;
    const int half = w >> 5, q = w & 31;
    const int i = ((q >> 2) - 4 * half) & 7, j = 4 * half + (q & 3);
    const int r = 8 * rb + i, col = 8 * cb + j;
    dst[d] = (r < rows && col < cols) ? src[c * (size_t)rows * ld + (size_t)r * ld + col] : 0.f;
  }
}

// TF32 split for the pipelined kernel: hi = x rounded to the TF32 grid (to
// nearest, ties away from zero: the same value as cvt.rna), lo = x - hi
// exactly, passed to the MMA as raw FP32 bits, of which the tensor core reads
// the TF32 part (|lo| <= 2^-11 |x|, so what is dropped is below 2^-21 |x|).
__device__ __forceinline__ void split_fast(float x, unsigned& hi, unsigned& lo) {
  hi = (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
  lo = __float_as_uint(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_split_a(float (&d)[4], const float (&a)[4], unsigned bh0, unsigned bh1,
                                            unsigned bl0, unsigned bl1) {
  unsigned ah[4], al[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) split_fast(a[i], ah[i], al[i]);
  mma_tf32(d, al, bh0, bh1);
  mma_tf32(d, ah, bl0, bl1);
  mma_tf32(d, ah, bh0, bh1);
}

__device__ __forceinline__ void mma_split_a_2acc(float (&dh)[4], float (&dl)[4], const float (&a)[4], unsigned bh0,
                                                 unsigned bh1, unsigned bl0, unsigned bl1) {
  unsigned ah[4], al[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) split_fast(a[i], ah[i], al[i]);
  mma_tf32(dl, al, bh0, bh1);
  mma_tf32(dl, ah, bl0, bl1);
  mma_tf32(dh, ah, bh0, bh1);
}

// One problem of the pipelined x-update: its stage layout, tables and spectra.
struct PipeProb {
  PipePlan P;
  const float* what_o;   // W_hat in the block layout [nclass][tm/8][zm/8][64]
  const float* hinv_o;   // H^-1 in the block layout [nclass][zm/8][zm/8][64]
  const float* lap;      // [nclass]
  const int* members;    // [nclass][4]
  int nclass;
  const float2* c_hat;   // [nf][ldt]
  const float2* s_hat;   // [nf][ldz]
  float2* x_hat;         // [nf][ldz] in / out
  float2* kx_hat;        // [nf][ldt] out
  int ldt, ldz;
  float inv_s;
  int item0;             // first work-queue item of this problem
};

// Producer: class c of problem q into stage `st` (header, then the bulk copies
// completing on `full`).
__device__ __forceinline__ void produce_item(const PipeProb& q, int c, unsigned char* st, uint64_t* full) {
  const PipePlan& P = q.P;
  int f[4];
  unsigned bytes = P.w_bytes + P.h_bytes;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    f[m] = __ldg(q.members + 4 * c + m);
    if (f[m] >= 0) bytes += P.c_bytes + 2 * P.v_bytes;
  }
  // the class header (members + 1, diagonal of L) for the consumers; the
  // arrive below releases these stores to them.  Header words stay small
  // non-negative integers or finite floats: in the many-problem kernel one
  // problem's header may sit inside another's operand padding, which is then
  // multiplied by zero.
  int* hdr = reinterpret_cast<int*>(st + P.o_hdr);
#pragma unroll
  for (int m = 0; m < 4; ++m) hdr[m] = f[m] + 1;
  reinterpret_cast<float*>(hdr)[4] = __ldg(q.lap + c) + 1.0f;
  mbar_expect_tx(full, bytes);
  bulk_g2s(st + P.o_w, q.what_o + (size_t)c * P.tm * P.zm, P.w_bytes, full);
  bulk_g2s(st + P.o_h, q.hinv_o + (size_t)c * P.zm * P.zm, P.h_bytes, full);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    if (f[m] < 0) continue;
    bulk_g2s(st + P.o_c + m * P.cs * 4, q.c_hat + (size_t)f[m] * q.ldt, P.c_bytes, full);
    bulk_g2s(st + P.o_s + m * P.sz * 4, q.s_hat + (size_t)f[m] * q.ldz, P.v_bytes, full);
    bulk_g2s(st + P.o_x + m * P.sz * 4, q.x_hat + (size_t)f[m] * q.ldz, P.v_bytes, full);
  }
}

// Scratch of the consumers (per CTA, sized for ZMX padded depths).
struct PipeScratch {
  float* part;     // [warp][ZM][8] adjoint partial sums
  unsigned* bh;    // [ZM][8] b, TF32 hi / raw lo
  unsigned* bl;
  unsigned* xh;    // [ZM][8] x_new, TF32 hi / raw lo
  unsigned* xl;
};

// Consumers (8 warps): the x-update of the class in stage `st`.  KZC > 0 fixes
// the forward K steps at compile time; KZC = 0 takes them from the problem
// (at most 8), with the same operations in the same order.  `gave_up` is this
// thread's full-barrier timeout; returns true when the CTA must stop.
template <int KZC>
__device__ __forceinline__ bool consume_item(const PipeProb& q, const unsigned char* st, const PipeScratch& scr,
                                             int gave_up) {
  constexpr int KZM = KZC > 0 ? KZC : 8;
  constexpr int MZM = (KZM + 1) / 2;
  const PipePlan& P = q.P;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, tg = lane & 3;
  const int hg = g >> 2;
  // word offsets of this lane's fragment elements inside an 8 x 8 block
  const int offF0 = 4 * g + tg;                                       // (row g, column tg)
  const int offF2 = 32 + 4 * ((g + 4) & 7) + tg;                      // (row g, column tg + 4)
  const int offA0 = 32 * hg + 4 * ((tg + 4 * hg) & 7) + (g & 3);      // (row tg, column g)
  const int offA2 = 32 * hg + 4 * ((tg + 4 + 4 * hg) & 7) + (g & 3);  // (row tg + 4, column g)
  const int nt = P.nt, nz = P.nz;
  const int KZ = KZC > 0 ? KZC : (nz + 7) >> 3;
  const int MZ = (KZ + 1) >> 1, ZB = 2 * MZ, ZM = 16 * MZ;
  const int kt = (nt + 7) >> 3, mtt = P.tm >> 4;
  const float inv_s = q.inv_s;
  const float* W = reinterpret_cast<const float*>(st + P.o_w);
  const float* H = reinterpret_cast<const float*>(st + P.o_h);
  const float* C = reinterpret_cast<const float*>(st + P.o_c);
  const float* SV = reinterpret_cast<const float*>(st + P.o_s);
  const float* XV = reinterpret_cast<const float*>(st + P.o_x);
  const int* hdr = reinterpret_cast<const int*>(st + P.o_hdr);

  // ---- A: adjoint partial sums y_w[z][r] = sum over this warp's t of W[t][z] c[t][r] ----
  {
    float acc[MZM][4];
#pragma unroll
    for (int mt = 0; mt < MZM; ++mt)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[mt][i] = 0.f;
    const float* cr = C + (g >> 1) * P.cs + 2 * tg + (g & 1) + 16 * warp;  // t = 8 ks + tg
    const float* wa0 = W + warp * ZB * 64 + offA0;
    const float* wa2 = W + warp * ZB * 64 + offA2;
#pragma unroll 2
    for (int ks = warp; ks < kt; ks += PIPE_CONS_WARPS) {
      unsigned bh0, bl0, bh1, bl1;
      split_fast(cr[0], bh0, bl0);
      split_fast(cr[8], bh1, bl1);
#pragma unroll
      for (int mt = 0; mt < MZM; ++mt) {
        if (mt < MZ) {
          const float a[4] = {wa0[128 * mt], wa0[128 * mt + 64], wa2[128 * mt], wa2[128 * mt + 64]};
          mma_split_a(acc[mt], a, bh0, bh1, bl0, bl1);
        }
      }
      cr += 16 * PIPE_CONS_WARPS;
      wa0 += PIPE_CONS_WARPS * ZB * 64;
      wa2 += PIPE_CONS_WARPS * ZB * 64;
    }
#pragma unroll
    for (int mt = 0; mt < MZM; ++mt) {
      if (mt < MZ) {
        float* p = scr.part + (warp * ZM + 16 * mt + g) * 8 + 2 * tg;
        *reinterpret_cast<float2*>(p) = make_float2(acc[mt][0], acc[mt][1]);
        *reinterpret_cast<float2*>(p + 64) = make_float2(acc[mt][2], acc[mt][3]);
      }
    }
  }
  if (cons_sync_or(gave_up)) return true;
  // ---- B: b = y / s + s_hat - L x_prev, split for the H^-1 MMA ----
  {
    const float dl = reinterpret_cast<const float*>(hdr)[4];
    for (int i = tid; i < nz * 8; i += PIPE_CONS_THREADS) {
      const int z = i >> 3, r = i & 7, m = r >> 1, cp = r & 1;
      float y = 0.f;
#pragma unroll
      for (int w = 0; w < PIPE_CONS_WARPS; ++w) y += scr.part[w * ZM * 8 + i];
      const float* xm = XV + m * P.sz + cp + 2 * z;
      const float xz = xm[0];
      float lx = dl * xz;
      if (z > 0) lx += xz - xm[-2];
      if (z < nz - 1) lx -= xm[2] - xz;
      unsigned h, l;
      split_fast(y * inv_s + SV[m * P.sz + 2 * z + cp] - lx, h, l);
      scr.bh[i] = h;
      scr.bl[i] = l;
    }
    // rows z in [nz, ZM) of b stay zero (this problem's padding)
    for (int i = nz * 8 + tid; i < ZM * 8; i += PIPE_CONS_THREADS) {
      scr.bh[i] = 0u;
      scr.bl[i] = 0u;
    }
  }
  cons_sync();
  const int mem_tg = hdr[tg] - 1;  // this lane's output member (D columns 2 tg, 2 tg + 1)
  // ---- C: x_new = x_prev + H^-1 b; one warp per 16-row z tile ----
  if (warp < MZ) {
    float ah[4] = {0.f, 0.f, 0.f, 0.f}, al[4] = {0.f, 0.f, 0.f, 0.f};
    const float* h0 = H + 2 * warp * ZB * 64;  // block (z / 8 = 2 warp, w / 8 = 0)
#pragma unroll
    for (int ks = 0; ks < 2 * MZM; ++ks) {
      if (ks < ZB) {
        const float* hb = h0 + ks * 64;
        const float a[4] = {hb[offF0], hb[ZB * 64 + offF0], hb[offF2], hb[ZB * 64 + offF2]};
        const int b0 = (8 * ks + tg) * 8 + g, b1 = b0 + 32;
        mma_split_a_2acc(ah, al, a, scr.bh[b0], scr.bh[b1], scr.bl[b0], scr.bl[b1]);
      }
    }
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      const int z = 16 * warp + g + 8 * hf;
      const float2 xp = z < nz ? *reinterpret_cast<const float2*>(XV + tg * P.sz + 2 * z) : make_float2(0.f, 0.f);
      const float2 xn = make_float2(xp.x + (ah[2 * hf] + al[2 * hf]), xp.y + (ah[2 * hf + 1] + al[2 * hf + 1]));
      if (z < nz && mem_tg >= 0) q.x_hat[(size_t)mem_tg * q.ldz + z] = xn;
      unsigned h0b, l0b, h1b, l1b;
      split_fast(xn.x, h0b, l0b);
      split_fast(xn.y, h1b, l1b);
      *reinterpret_cast<uint2*>(scr.xh + z * 8 + 2 * tg) = make_uint2(h0b, h1b);
      *reinterpret_cast<uint2*>(scr.xl + z * 8 + 2 * tg) = make_uint2(l0b, l1b);
    }
  }
  cons_sync();
  // ---- D: Kx[t][r] = sum_z W[t][z] x_new[z][r] / s; each warp two 16-row t tiles at a time ----
  {
    unsigned xb[KZM][4];  // B fragments (hi0, hi1, lo0, lo1) of every K step, shared by the tiles
#pragma unroll
    for (int ks = 0; ks < KZM; ++ks) {
      if (ks < KZ) {
        const int b0 = (8 * ks + tg) * 8 + g;
        xb[ks][0] = scr.xh[b0];
        xb[ks][1] = scr.xh[b0 + 32];
        xb[ks][2] = scr.xl[b0];
        xb[ks][3] = scr.xl[b0 + 32];
      }
    }
    float2* dst = mem_tg >= 0 ? q.kx_hat + (size_t)mem_tg * q.ldt : nullptr;
    for (int mt = warp; mt < mtt; mt += 2 * PIPE_CONS_WARPS) {
      const int mt2 = mt + PIPE_CONS_WARPS;
      const bool two = mt2 < mtt;
      float dh[2][4] = {}, dlo[2][4] = {};
      const float* w0 = W + 2 * mt * ZB * 64;  // block (t / 8 = 2 mt, z / 8 = 0)
      const float* w1 = W + 2 * mt2 * ZB * 64;
#pragma unroll
      for (int ks = 0; ks < KZM; ++ks) {
        if (ks < KZ) {
          const float a0[4] = {w0[ks * 64 + offF0], w0[(ZB + ks) * 64 + offF0], w0[ks * 64 + offF2],
                               w0[(ZB + ks) * 64 + offF2]};
          mma_split_a_2acc(dh[0], dlo[0], a0, xb[ks][0], xb[ks][1], xb[ks][2], xb[ks][3]);
          if (two) {
            const float a1[4] = {w1[ks * 64 + offF0], w1[(ZB + ks) * 64 + offF0], w1[ks * 64 + offF2],
                                 w1[(ZB + ks) * 64 + offF2]};
            mma_split_a_2acc(dh[1], dlo[1], a1, xb[ks][0], xb[ks][1], xb[ks][2], xb[ks][3]);
          }
        }
      }
      if (dst) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if (u == 1 && !two) break;
          const int t = 16 * (u ? mt2 : mt) + g;
          if (t < nt) dst[t] = make_float2((dh[u][0] + dlo[u][0]) * inv_s, (dh[u][1] + dlo[u][1]) * inv_s);
          if (t + 8 < nt) dst[t + 8] = make_float2((dh[u][2] + dlo[u][2]) * inv_s, (dh[u][3] + dlo[u][3]) * inv_s);
        }
      }
    }
  }
  return false;
}

// Shared set-up of both pipelined kernels: zero `zero_bytes` of shared memory
// (operand padding then reads as zeros), initialise the stage barriers.
__device__ __forceinline__ void pipe_setup(unsigned char* sm, int zero_bytes, uint64_t* full, uint64_t* empty, int S,
                                           volatile int* s_abort) {
  for (int i = threadIdx.x; i < zero_bytes / 16; i += PIPE_THREADS)
    reinterpret_cast<float4*>(sm)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, PIPE_CONS_WARPS);
    }
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // zeroes before the bulk copies
  __syncthreads();
}

// Producer wait for a free stage: bounded, and it stops early once the
// consumers have given up.  Returns false (after flagging a timeout of its
// own) when no more stages must be filled.
__device__ __forceinline__ bool wait_free(uint64_t* empty, uint32_t par, long long max_polls, volatile int* s_abort,
                                          int* status_flag) {
  for (long long i = 0; i < max_polls; ++i) {
    if (mbar_try(empty, par)) return true;
    if (*s_abort) return false;
  }
  if (!*s_abort) {
    atomicExch(status_flag, 1);
    *s_abort = 1;
  }
  return false;
}

// No copy may be in flight when the CTA exits: wait for each stage's last fill.
__device__ __forceinline__ void drain_fills(uint64_t* full, int S, int issued) {
  for (int s = 0; s < S; ++s) {
    if (issued > s) {
      const int last = s + ((issued - 1 - s) / S) * S;
      mbar_wait_bounded(full + s, (uint32_t)((last / S) & 1), PIPE_DRAIN_POLLS);
    }
  }
}

// Single problem: CTA b takes classes b, b + grid, ...
// KZ = forward K steps = ceil(nz / 8); MZ = 16-row z tiles = ceil(nz / 16).
template <int KZ>
__global__ void __launch_bounds__(PIPE_THREADS, 1) k_contract_admm_pipe(PipeProb q, int* status_flag,
                                                                        long long max_polls) {
  extern __shared__ __align__(128) float4 sm_pipe[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(sm_pipe);
  const PipePlan& P = q.P;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = P.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + P.o_bar);
  uint64_t* empty = full + S;
  volatile int* s_abort = reinterpret_cast<volatile int*>(empty + S);
  pipe_setup(sm, P.o_bar, full, empty, S, s_abort);
  const int nclass = q.nclass;
  const int mine = (int)blockIdx.x < nclass ? (nclass - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (warp == PIPE_CONS_WARPS) {
    if (lane != 0) return;
    int issued = 0;
    for (; issued < mine; ++issued) {
      const int s = issued % S;
      if (!wait_free(empty + s, ((issued / S) & 1) ^ 1, max_polls, s_abort, status_flag)) break;
      produce_item(q, (int)blockIdx.x + issued * (int)gridDim.x, sm + s * P.stage_bytes, full + s);
    }
    drain_fills(full, S, issued);
    return;
  }
  const PipeScratch scr{reinterpret_cast<float*>(sm + P.o_part), reinterpret_cast<unsigned*>(sm + P.o_bh),
                        reinterpret_cast<unsigned*>(sm + P.o_bl), reinterpret_cast<unsigned*>(sm + P.o_xh),
                        reinterpret_cast<unsigned*>(sm + P.o_xl)};
  for (int k = 0; k < mine; ++k) {
    const int s = k % S;
    int gave_up = 0;
    if (!mbar_wait_bounded(full + s, (uint32_t)((k / S) & 1), max_polls)) {
      gave_up = 1;
      atomicExch(status_flag, 1);
    }
    if (consume_item<KZ>(q, sm + s * P.stage_bytes, scr, gave_up)) {
      if (threadIdx.x == 0) *s_abort = 1;
      break;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty + s);
  }
}

// Many problems, one persistent launch: the producer of each CTA takes items
// (problem, class) from a device work queue (an atomic counter, QCHUNK items
// per grab; problems in the queue in the caller's order, largest class blocks
// first), so that CTAs done with one problem's classes go on with the next.
// Stages are sized for the largest problem plus a 32-byte tail whose first
// word names the item's problem + 1 (0: the queue is empty, the consumers stop).
constexpr int QCHUNK = 8;

__global__ void __launch_bounds__(PIPE_THREADS, 1) k_contract_admm_queue(const PipeProb* __restrict__ probs, int nprob,
                                                                         int total, int* queue, int stage_bytes,
                                                                         int S, int o_scr, int zm_max,
                                                                         int* status_flag, long long max_polls) {
  extern __shared__ __align__(128) float4 sm_pipe[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(sm_pipe);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // layout: S stages | consumer scratch | problem table | barriers
  const int o_part = o_scr, o_bh = o_part + PIPE_CONS_WARPS * zm_max * 32, o_bl = o_bh + zm_max * 32,
            o_xh = o_bl + zm_max * 32, o_xl = o_xh + zm_max * 32, o_tab = o_xl + zm_max * 32;
  PipeProb* tab = reinterpret_cast<PipeProb*>(sm + o_tab);
  const int o_bar = o_tab + ((nprob * (int)sizeof(PipeProb) + 15) & ~15);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + o_bar);
  uint64_t* empty = full + S;
  volatile int* s_abort = reinterpret_cast<volatile int*>(empty + S);
  for (int i = threadIdx.x; i < nprob * (int)sizeof(PipeProb) / 4; i += PIPE_THREADS)
    reinterpret_cast<int*>(tab)[i] = reinterpret_cast<const int*>(probs)[i];
  pipe_setup(sm, o_tab, full, empty, S, s_abort);
  if (warp == PIPE_CONS_WARPS) {
    if (lane != 0) return;
    int issued = 0, cur = 0, end = 0, pi = 0;
    for (;;) {
      if (cur >= end) {
        cur = atomicAdd(queue, QCHUNK);
        end = min(cur + QCHUNK, total);
      }
      const bool more = cur < total;
      const int s = issued % S;
      if (!wait_free(empty + s, ((issued / S) & 1) ^ 1, max_polls, s_abort, status_flag)) break;
      unsigned char* st = sm + s * stage_bytes;
      int* slot = reinterpret_cast<int*>(st + stage_bytes - 16);  // the item's problem + 1, 0 = queue empty
      if (!more) {
        *slot = 0;
        mbar_arrive(full + s);
        ++issued;
        break;
      }
      while (pi + 1 < nprob && tab[pi + 1].item0 <= cur) ++pi;  // items come in increasing order
      *slot = pi + 1;
      produce_item(tab[pi], cur - tab[pi].item0, st, full + s);
      ++cur;
      ++issued;
    }
    drain_fills(full, S, issued);
    return;
  }
  const PipeScratch scr{reinterpret_cast<float*>(sm + o_part), reinterpret_cast<unsigned*>(sm + o_bh),
                        reinterpret_cast<unsigned*>(sm + o_bl), reinterpret_cast<unsigned*>(sm + o_xh),
                        reinterpret_cast<unsigned*>(sm + o_xl)};
  for (int k = 0;; ++k) {
    const int s = k % S;
    int gave_up = 0;
    if (!mbar_wait_bounded(full + s, (uint32_t)((k / S) & 1), max_polls)) {
      gave_up = 1;
      atomicExch(status_flag, 1);
    }
    const unsigned char* st = sm + s * stage_bytes;
    const int pi = *reinterpret_cast<const int*>(st + stage_bytes - 16) - 1;
    if (cons_sync_or(gave_up)) {
      if (threadIdx.x == 0) *s_abort = 1;
      break;
    }
    if (pi < 0) break;
    if (consume_item<0>(tab[pi], st, scr, 0)) {
      if (threadIdx.x == 0) *s_abort = 1;
      break;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty + s);
  }
}

template <int KZ>
ctof_status launch_pipe(const ctof_kernel_s* k, const PipePlan& P, int grid, const float2* c_hat, const float2* s_hat,
                        float2* x_hat, float2* kx_hat, float inv_scale, cudaStream_t st) {
  CTOF_CUDA_TRY(
      cudaFuncSetAttribute(k_contract_admm_pipe<KZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, P.total));
  PipeProb q{};
  q.P = P;
  q.what_o = k->d_what_admm;
  q.hinv_o = k->d_hinv_admm;
  q.lap = k->d_lap;
  q.members = k->d_members;
  q.nclass = k->nclass;
  q.c_hat = c_hat;
  q.s_hat = s_hat;
  q.x_hat = x_hat;
  q.kx_hat = kx_hat;
  q.ldt = k->ldt;
  q.ldz = k->ldz;
  q.inv_s = inv_scale;
  q.item0 = 0;
  k_contract_admm_pipe<KZ><<<grid, PIPE_THREADS, P.total, st>>>(q, k->d_flags, k->max_polls);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

}  // namespace

size_t contract_admm_smem_bytes(int nt, int nz, int nbuf) { return (size_t)make_layout(nt, nz, nbuf).total_floats * 4; }

int contract_admm_pipe_stages(int nt, int nz) { return pipe_stages(nt, nz); }

size_t contract_admm_pipe_floats(int nt, int nz, int which) {
  if (!pipe_stages(nt, nz)) return 0;
  const size_t tm = (size_t)rup(nt, 16), zm = (size_t)rup(nz, 16);
  return which == 0 ? tm * zm : zm * zm;
}

ctof_status contract_admm_prepare(ctof_kernel_s* k, cudaStream_t st) {
  if (!k->d_what_admm || !k->d_hinv_admm) return CTOF_OK;
  const int tm = rup(k->nt, 16), zm = rup(k->nz, 16);
  k_admm_reorder<<<152 * 8, 256, 0, st>>>(k->d_what, k->nt, k->nz, k->z4, tm, zm, k->d_what_admm, k->nclass);
  CTOF_CUDA_TRY(cudaGetLastError());
  k_admm_reorder<<<152 * 8, 256, 0, st>>>(k->d_hinv, k->nz, k->nz, k->z4, zm, zm, k->d_hinv_admm, k->nclass);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status contract_admm(const ctof_kernel_s* k, const float2* c_hat, const float2* s_hat, float2* x_hat,
                          float2* kx_hat, float inv_scale, cudaStream_t st) {
  const int stages = k->d_what_admm ? pipe_stages(k->nt, k->nz) : 0;
  if (stages) {
    const PipePlan P = make_pipe_plan(k->nt, k->nz, stages);
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, k->device);
    const int grid = k->nclass < nsm ? k->nclass : nsm;
    switch ((k->nz + 7) >> 3) {
      case 1: return launch_pipe<1>(k, P, grid, c_hat, s_hat, x_hat, kx_hat, inv_scale, st);
      case 2: return launch_pipe<2>(k, P, grid, c_hat, s_hat, x_hat, kx_hat, inv_scale, st);
      case 3: return launch_pipe<3>(k, P, grid, c_hat, s_hat, x_hat, kx_hat, inv_scale, st);
      case 4: return launch_pipe<4>(k, P, grid, c_hat, s_hat, x_hat, kx_hat, inv_scale, st);
      case 5: return launch_pipe<5>(k, P, grid, c_hat, s_hat, x_hat, kx_hat, inv_scale, st);
      case 6: return launch_pipe<6>(k, P, grid, c_hat, s_hat, x_hat, kx_hat, inv_scale, st);
      case 7: return launch_pipe<7>(k, P, grid, c_hat, s_hat, x_hat, kx_hat, inv_scale, st);
      default: return launch_pipe<8>(k, P, grid, c_hat, s_hat, x_hat, kx_hat, inv_scale, st);
    }
  }
  const size_t limit = 227 * 1024;
  // Two single-buffered CTAs per SM when they fit (one computes while the
  // other loads), else one double-buffered CTA.
  int per_sm = 2;
  AdmmLayout L = make_layout(k->nt, k->nz, 1);
  if (2 * ((size_t)L.total_floats * 4 + 1024) > 228 * 1024) {
    per_sm = 1;
    L = make_layout(k->nt, k->nz, 2);
    if ((size_t)L.total_floats * 4 > limit) L = make_layout(k->nt, k->nz, 1);
  }
  if ((size_t)L.total_floats * 4 > limit) return CTOF_EUNSUPPORTED;
  const size_t sm = (size_t)L.total_floats * 4;
  CTOF_CUDA_TRY(cudaFuncSetAttribute(k_contract_admm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, k->device);
  const int grid = k->nclass < per_sm * nsm ? k->nclass : per_sm * nsm;
  k_contract_admm<<<grid, AD_THREADS, sm, st>>>(L, k->d_what, k->d_hinv, k->d_lap, k->d_members, k->nclass, c_hat,
                                                k->ldt, s_hat, x_hat, k->ldz, kx_hat, inv_scale);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

// ---- many problems in one persistent launch --------------------------------

namespace {

struct QueueLayout {
  int stage_bytes, stages, o_scr, zm_max, smem;
};

QueueLayout queue_layout(int max_layout, int zm_max, int nprob, int stages) {
  QueueLayout L;
  L.stage_bytes = rup(max_layout + 32, 128);
  L.stages = stages;
  L.zm_max = zm_max;
  L.o_scr = stages * L.stage_bytes;
  const int scratch = PIPE_CONS_WARPS * zm_max * 32 + 4 * zm_max * 32;
  const int table = (nprob * (int)sizeof(PipeProb) + 15) & ~15;
  L.smem = L.o_scr + scratch + table + 2 * stages * 8 + 16;
  return L;
}

// The device work-queue counter sits after the problem table.
size_t queue_counter_offset(int nprob) { return ((size_t)nprob * sizeof(PipeProb) + 255) & ~(size_t)255; }

}  // namespace

ctof_status admm_queue_build(int count, ctof_kernel_s* const* ks, AdmmQueue* out) {
  admm_queue_free(out);
  struct Cand {
    int idx, layout, zm;
  };
  std::vector<Cand> cand;
  for (int i = 0; i < count; ++i) {
    const ctof_kernel_s* k = ks[i];
    if (!k->d_what_admm || !pipe_stages(k->nt, k->nz)) continue;
    const PipePlan P = make_pipe_plan(k->nt, k->nz, 2);
    cand.push_back({i, P.stage_bytes, P.zm});
  }
  // the largest set, taken from the smallest class blocks up, whose two stages fit
  std::sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) { return a.layout < b.layout; });
  int take = 0, max_layout = 0, zm_max = 16;
  for (int j = 0; j < (int)cand.size(); ++j) {
    const int ml = std::max(max_layout, cand[j].layout), zm = std::max(zm_max, cand[j].zm);
    if (queue_layout(ml, zm, j + 1, 2).smem > PIPE_SMEM_LIMIT) break;
    max_layout = ml;
    zm_max = zm;
    take = j + 1;
  }
  if (take < 2) return CTOF_OK;  // nothing to gain: every problem keeps its own launch
  cand.resize(take);
  // queue order: largest class blocks first, so that small ones fill in at the end
  std::sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) { return a.layout > b.layout; });
  int stages = 2;
  while (stages < 4 && queue_layout(max_layout, zm_max, take, stages + 1).smem <= PIPE_SMEM_LIMIT) ++stages;
  const QueueLayout L = queue_layout(max_layout, zm_max, take, stages);
  std::vector<PipeProb> tab(take);
  int items = 0;
  for (int j = 0; j < take; ++j) {
    const ctof_kernel_s* k = ks[cand[j].idx];
    PipeProb& q = tab[j];
    q.P = make_pipe_plan(k->nt, k->nz, 2);
    q.what_o = k->d_what_admm;
    q.hinv_o = k->d_hinv_admm;
    q.lap = k->d_lap;
    q.members = k->d_members;
    q.nclass = k->nclass;
    q.c_hat = k->d_spec_t2;
    q.s_hat = k->d_spec_z;
    q.x_hat = k->d_spec_z2;
    q.kx_hat = k->d_spec_t;
    q.ldt = k->ldt;
    q.ldz = k->ldz;
    q.inv_s = (float)(1.0 / k->scale);
    q.item0 = items;
    items += k->nclass;
  }
  void* d = nullptr;
  const size_t tbytes = (size_t)take * sizeof(PipeProb);
  if (cudaMalloc(&d, queue_counter_offset(take) + 256) != cudaSuccess) {
    cudaGetLastError();
    return CTOF_ENOMEM;
  }
  out->d_mem = d;
  if (cudaMemcpy(d, tab.data(), tbytes, cudaMemcpyHostToDevice) != cudaSuccess) {
    admm_queue_free(out);
    return CTOF_ECUDA;
  }
  for (int j = 0; j < take; ++j) out->members.push_back(cand[j].idx);
  out->nprob = take;
  out->total = items;
  out->stage_bytes = L.stage_bytes;
  out->stages = L.stages;
  out->o_scr = L.o_scr;
  out->zm_max = L.zm_max;
  out->smem = L.smem;
  out->flag = ks[cand[0].idx]->d_flags;
  out->max_polls = ks[cand[0].idx]->max_polls;
  out->nsm = 152;
  cudaDeviceGetAttribute(&out->nsm, cudaDevAttrMultiProcessorCount, ks[cand[0].idx]->device);
  return CTOF_OK;
}

ctof_status admm_queue_launch(const AdmmQueue& q, cudaStream_t st) {
  if (q.nprob == 0) return CTOF_OK;
  const PipeProb* tab = static_cast<const PipeProb*>(q.d_mem);
  int* ctr = reinterpret_cast<int*>(static_cast<char*>(q.d_mem) + queue_counter_offset(q.nprob));
  CTOF_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(int), st));
  CTOF_CUDA_TRY(cudaFuncSetAttribute(k_contract_admm_queue, cudaFuncAttributeMaxDynamicSharedMemorySize, q.smem));
  k_contract_admm_queue<<<q.nsm, PIPE_THREADS, q.smem, st>>>(tab, q.nprob, q.total, ctr, q.stage_bytes, q.stages,
                                                            q.o_scr, q.zm_max, q.flag, q.max_polls);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

void admm_queue_free(AdmmQueue* q) {
  if (q->d_mem) cudaFree(q->d_mem);
  q->d_mem = nullptr;
  q->nprob = 0;
  q->total = 0;
  q->members.clear();
}
