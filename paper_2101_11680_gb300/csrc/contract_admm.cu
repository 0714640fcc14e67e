// Fused ADMM x-update per frequency class (Eq. 11 in the lateral Fourier
// domain, one iteration of the normal-equation solve):
//   b     = W_hat^T c_hat / s + s_hat - L x_hat_prev          (Z x 8 real)
//   x_hat = x_hat_prev + H^-1 b
//   Kx    = W_hat x_hat / s                                     (T x 8 real)
// with L = (|dx|^2 + |dy|^2 + 1) I + Dz^T Dz and H = W_hat^T W_hat / s^2 + L,
// i.e. x_hat = H^-1 (W_hat^T (K x_hat_prev + c_hat)/s + s_hat).  The 8 real
// right-hand sides are the real/imaginary parts of the up-to-4 frequencies
// of one class (they share the real matrix W_hat).
//
// The kernel streams W_hat once per iteration.  Persistent CTAs of 8 warps walk
// the classes, two per SM where their shared memory fits (one buffer each: the
// phases of one class run between block-wide barriers, and the other CTA's
// class fills the SM meanwhile); otherwise one CTA per SM prefetches class
// i+1 (W_hat block, H^-1 block and the member vectors) with 16-byte cp.async
// copies into the second of two shared-memory buffers.
// (Per-row TMA bulk copies were measured slower here: 300+ requests of 192
// bytes per class are limited by the TMA request rate, not by bandwidth.)
// The two T x Z contractions run on the warp-level tensor-core MMA
// (m16n8k8, TF32 inputs, FP32 accumulation) with each operand split into a
// TF32 high part and a TF32 remainder (three MMAs per tile: lo*hi + hi*lo +
// hi*hi), which keeps FP32-level accuracy; N = 8 is exactly the 8 real
// right-hand sides of a class.  Shared W_hat rows are padded to a stride zp
// with zp/4 odd so that the MMA fragment loads hit distinct banks.
//   adjoint part: warps split the t (K) steps over all z tiles; partial
//                 results meet in shared memory.
//   H^-1 part:    FP32 FMA, thread per (z, member).
//   forward part: one warp per 16-row tile of t.
#include <cuda_runtime.h>

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

}  // namespace

size_t contract_admm_smem_bytes(int nt, int nz, int nbuf) { return (size_t)make_layout(nt, nz, nbuf).total_floats * 4; }

ctof_status contract_admm(const ctof_kernel_s* k, const float2* c_hat, const float2* s_hat, float2* x_hat,
                          float2* kx_hat, float inv_scale, cudaStream_t st) {
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
