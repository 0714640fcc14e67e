// Precision form: Tikhonov reconstruction of a batch of B measurement volumes
// that share one kernel, with the per-frequency contraction b = W_hat^T m_hat
// on BF16 tensor cores and mixed-precision iterative refinement of the
// Z x Z solve (the regularised inverse of Eq. 7 per lateral frequency).
//
//   W_hat = Q_hi + Q_lo,  m_hat = M_hi + M_lo        (BF16 pairs, exact split)
//   b0    = Q_hi^T M_hi                              (one BF16 GEMM term)
//   b     = Q_hi^T M_hi + Q_hi^T M_lo + Q_lo^T M_hi  (three terms, FP32 accumulation)
//   x0    = C b0,   x_{i+1} = x_i + C (b - (G + lambda I) x_i)
// with C = (G + lambda I)^-1 (FP64 Cholesky, stored FP32) and G the FP64 Gram
// (stored FP32 for the residual).  x0 carries the BF16 error; each refinement
// step replaces it by the error of the three-term product (about 2^-16).
//
// One CTA (8 warps) per frequency class at a time: Q_hi / Q_lo (T x Zs, Zs the
// depth count rounded to 16/32/64) and C, G stay in shared memory while the
// batch streams through in chunks of two volumes (8 members x 2 volumes = 16
// real right-hand sides).  Fragments come from swizzled shared rows via
// ldmatrix (Q^T through .trans); products use mma.sync m16n8k16 BF16.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

#include "ctof_internal.h"

namespace {

constexpr int BT_THREADS = 256;
constexpr int BT_WARPS = BT_THREADS / 32;
constexpr int BC = 2;            // volumes per chunk
constexpr int NB = 8 * BC;       // real right-hand sides per chunk

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void ldsm_x4_trans(unsigned (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2(unsigned (&r)[2], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct BtLayout {
  int nt, nz, z4, zs, tk;  // tk = nt rounded up to 16 (K extent)
  int cs;                  // shared row pitch of C and G + lambda I: 4 (z4/4 | 1) floats
  int batch;
  // byte offsets in shared memory
  int off_qh, off_ql, off_mh, off_ml, off_c, off_g, off_b0, off_bf, off_x;
  int total;
};

// Q rows: zs bf16 = zs/8 chunks, chunk index XOR (t & (zs/8 - 1)).
__device__ __forceinline__ int q_off(const BtLayout& L, int t, int chunk) {
  const int mask = (L.zs >> 3) - 1;
  return (t * L.zs + ((chunk ^ (t & mask)) << 3)) * 2;
}
// M rows (one per right-hand side n): tk bf16 = tk/8 chunks, chunk index rotated
// by (n & 7) modulo the chunk count (stays inside the row for any tk).
__device__ __forceinline__ int m_off(const BtLayout& L, int n, int chunk) {
  const int nch = L.tk >> 3;
  int cc = chunk + (n & 7);
  cc = cc >= nch ? cc - nch : cc;
  cc = cc >= nch ? cc % nch : cc;
  return (n * L.tk + (cc << 3)) * 2;
}

// sum_w row[w] v[w][nq .. nq+3] for v [.][NB] (FP32)
__device__ __forceinline__ float4 small_mv(const float* __restrict__ row, const float* __restrict__ v, int nz, int nq) {
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
  for (int w = 0; w < nz; ++w) {
    const float c = row[w];
    const float4 b = *reinterpret_cast<const float4*>(v + w * NB + nq);
    a.x = fmaf(c, b.x, a.x);
    a.y = fmaf(c, b.y, a.y);
    a.z = fmaf(c, b.z, a.z);
    a.w = fmaf(c, b.w, a.w);
  }
  return a;
}

__global__ void __launch_bounds__(BT_THREADS, 1) k_batch_tikhonov_bf16(
    BtLayout L, const __nv_bfloat16* __restrict__ qhi, const __nv_bfloat16* __restrict__ qlo,
    const float* __restrict__ cinv, const float* __restrict__ glam, const int* __restrict__ members, int nclass,
    const float2* __restrict__ m_hat, int ldm, float2* __restrict__ x_hat, int ldx, int refine) {
  extern __shared__ __align__(128) unsigned char smb[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, tg = lane & 3;
  const int nt = L.nt, nz = L.nz, zs = L.zs, tk = L.tk;
  float* s_c = reinterpret_cast<float*>(smb + L.off_c);    // [nz][cs]
  float* s_g = reinterpret_cast<float*>(smb + L.off_g);    // [nz][cs]
  float* s_b0 = reinterpret_cast<float*>(smb + L.off_b0);  // [zs][NB]
  float* s_bf = reinterpret_cast<float*>(smb + L.off_bf);  // [zs][NB]
  float* s_x = reinterpret_cast<float*>(smb + L.off_x);    // [zs][NB]
  // zero everything once: Q rows beyond nt, M rows beyond nt / absent members stay 0
  for (int i = tid * 16; i < L.total; i += BT_THREADS * 16)
    *reinterpret_cast<uint4*>(smb + i) = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  const int mtiles = zs >> 4, ksteps = tk >> 4;
  const int chunks_q = zs >> 3;
  for (int c = blockIdx.x; c < nclass; c += gridDim.x) {
    int mem[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) mem[m] = members[c * 4 + m];
    // ---- class tables: Q_hi, Q_lo (swizzled rows), C, G + lambda I ----
    {
      const __nv_bfloat16* qh = qhi + (size_t)c * nt * zs;
      const __nv_bfloat16* ql = qlo + (size_t)c * nt * zs;
      for (int i = tid; i < nt * chunks_q; i += BT_THREADS) {
        const int t = i / chunks_q, ch = i - t * chunks_q;
        cp_async16(smb + L.off_qh + q_off(L, t, ch), qh + (size_t)t * zs + ch * 8);
        cp_async16(smb + L.off_ql + q_off(L, t, ch), ql + (size_t)t * zs + ch * 8);
      }
      const int cq = L.z4 >> 2;
      for (int i = tid; i < nz * cq; i += BT_THREADS) {
        const int r = i / cq, ch = i - r * cq;
        cp_async16(s_c + r * L.cs + ch * 4, cinv + ((size_t)c * nz + r) * L.z4 + ch * 4);
        cp_async16(s_g + r * L.cs + ch * 4, glam + ((size_t)c * nz + r) * L.z4 + ch * 4);
      }
      cp_async_commit();
      cp_async_wait_all();
    }
    __syncthreads();
    for (int b0 = 0; b0 < L.batch; b0 += BC) {
      // ---- right-hand sides of this chunk, split into BF16 hi/lo, rows n = (m*BC + bl)*2 + comp ----
      {
        const int tch = tk >> 3;  // 8-sample chunks along t
        for (int i = tid; i < 4 * BC * tch; i += BT_THREADS) {
          const int ch = i % tch, mb = i / tch, bl = mb % BC, m = mb / BC;
          const int b = b0 + bl;
          const int n = (m * BC + bl) * 2;
          uint4 rh, rl, ih, il;
          unsigned* prh = reinterpret_cast<unsigned*>(&rh);
          unsigned* prl = reinterpret_cast<unsigned*>(&rl);
          unsigned* pih = reinterpret_cast<unsigned*>(&ih);
          unsigned* pil = reinterpret_cast<unsigned*>(&il);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
            const int t = ch * 8 + 2 * j;
            if (mem[m] >= 0 && b < L.batch) {
              const float2* src = m_hat + (size_t)mem[m] * ldm + (size_t)b * nt;
              if (t < nt) v0 = src[t];
              if (t + 1 < nt) v1 = src[t + 1];
            }
            const __nv_bfloat16 h0 = __float2bfloat16_rn(v0.x), h1 = __float2bfloat16_rn(v1.x);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(v0.x - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(v1.x - __bfloat162float(h1));
            const __nv_bfloat16 g0 = __float2bfloat16_rn(v0.y), g1 = __float2bfloat16_rn(v1.y);
            const __nv_bfloat16 k0 = __float2bfloat16_rn(v0.y - __bfloat162float(g0));
            const __nv_bfloat16 k1 = __float2bfloat16_rn(v1.y - __bfloat162float(g1));
            __nv_bfloat162 p;
            p.x = h0; p.y = h1; prh[j] = *reinterpret_cast<unsigned*>(&p);
            p.x = l0; p.y = l1; prl[j] = *reinterpret_cast<unsigned*>(&p);
            p.x = g0; p.y = g1; pih[j] = *reinterpret_cast<unsigned*>(&p);
            p.x = k0; p.y = k1; pil[j] = *reinterpret_cast<unsigned*>(&p);
          }
          *reinterpret_cast<uint4*>(smb + L.off_mh + m_off(L, n, ch)) = rh;
          *reinterpret_cast<uint4*>(smb + L.off_ml + m_off(L, n, ch)) = rl;
          *reinterpret_cast<uint4*>(smb + L.off_mh + m_off(L, n + 1, ch)) = ih;
          *reinterpret_cast<uint4*>(smb + L.off_ml + m_off(L, n + 1, ch)) = il;
        }
      }
      __syncthreads();
      // ---- b0 = Q_hi^T M_hi,  b = b0 + Q_hi^T M_lo + Q_lo^T M_hi ----
      for (int pair = warp; pair < mtiles * (NB / 8); pair += BT_WARPS) {
        const int mt = pair % mtiles, ntile = pair / mtiles;
        const int z0 = mt * 16, n0 = ntile * 8;
        float acc_h[4] = {0.f, 0.f, 0.f, 0.f}, acc_x[4] = {0.f, 0.f, 0.f, 0.f};
        const int jm = lane >> 3, r8 = lane & 7;
        for (int ks = 0; ks < ksteps; ++ks) {
          const int k0 = ks * 16;
          // A = Q^T tile (z0.., k0..): matrix jm = (t block jm>>1, z block jm&1)
          const int tq = k0 + ((jm >> 1) << 3) + r8;
          const int zc = (z0 >> 3) + (jm & 1);
          unsigned ah[4], al[4];
          ldsm_x4_trans(ah, smb + L.off_qh + q_off(L, tq, zc));
          ldsm_x4_trans(al, smb + L.off_ql + q_off(L, tq, zc));
          // B = M tile (k0.., n0..): matrix (lane>>3)&1 = t block, row = n
          const int nr = n0 + r8;
          const int tcn = (k0 >> 3) + ((lane >> 3) & 1);
          unsigned bh[2], bl[2];
          ldsm_x2(bh, smb + L.off_mh + m_off(L, nr, tcn));
          ldsm_x2(bl, smb + L.off_ml + m_off(L, nr, tcn));
          mma_bf16(acc_h, ah, bh);
          mma_bf16(acc_x, ah, bl);
          mma_bf16(acc_x, al, bh);
        }
        const int zr = z0 + g, nc = n0 + 2 * tg;
        s_b0[zr * NB + nc] = acc_h[0];
        s_b0[zr * NB + nc + 1] = acc_h[1];
        s_b0[(zr + 8) * NB + nc] = acc_h[2];
        s_b0[(zr + 8) * NB + nc + 1] = acc_h[3];
        s_bf[zr * NB + nc] = acc_h[0] + acc_x[0];
        s_bf[zr * NB + nc + 1] = acc_h[1] + acc_x[1];
        s_bf[(zr + 8) * NB + nc] = acc_h[2] + acc_x[2];
        s_bf[(zr + 8) * NB + nc + 1] = acc_h[3] + acc_x[3];
      }
      __syncthreads();
      // ---- x0 = C b0, then x += C (b - (G + lambda I) x) ----
      // Each thread owns one depth z and four right-hand sides: four independent
      // accumulators per row walk, rows of C and G at a pitch that puts the
      // eight depths of a warp on distinct banks.
      const int zq = tid >> 2, nq = (tid & 3) * 4;
      const bool own = zq < nz && tid < 4 * nz;
      if (own) {
        const float4 y = small_mv(s_c + zq * L.cs, s_b0, nz, nq);
        *reinterpret_cast<float4*>(s_x + zq * NB + nq) = y;
      }
      __syncthreads();
      for (int it = 0; it < refine; ++it) {
        if (own) {  // residual r = b - (G + lambda I) x into s_b0
          const float4 gx = small_mv(s_g + zq * L.cs, s_x, nz, nq);
          const float4 bf = *reinterpret_cast<const float4*>(s_bf + zq * NB + nq);
          *reinterpret_cast<float4*>(s_b0 + zq * NB + nq) =
              make_float4(bf.x - gx.x, bf.y - gx.y, bf.z - gx.z, bf.w - gx.w);
        }
        __syncthreads();
        if (own) {  // x += C r (each thread updates only its own entries)
          const float4 cr = small_mv(s_c + zq * L.cs, s_b0, nz, nq);
          float4* xp = reinterpret_cast<float4*>(s_x + zq * NB + nq);
          const float4 x = *xp;
          *xp = make_float4(x.x + cr.x, x.y + cr.y, x.z + cr.z, x.w + cr.w);
        }
        __syncthreads();
      }
      // ---- x_hat[f][b*nz + z] ----
      for (int i = tid; i < 4 * BC * nz; i += BT_THREADS) {
        const int z = i % nz, mb = i / nz, bl = mb % BC, m = mb / BC;
        const int b = b0 + bl;
        if (mem[m] < 0 || b >= L.batch) continue;
        const int n = (m * BC + bl) * 2;
        x_hat[(size_t)mem[m] * ldx + (size_t)b * nz + z] = make_float2(s_x[z * NB + n], s_x[z * NB + n + 1]);
      }
      __syncthreads();
    }
  }
}

// Q_hi / Q_lo tables from the FP32 W_hat ([c][t][z4] -> [c][t][zs], zero padded).
__global__ void k_split_bf16(const float* __restrict__ what, long long rows, int nz, int z4, int zs,
                             __nv_bfloat16* __restrict__ qhi, __nv_bfloat16* __restrict__ qlo) {
  const long long n = rows * zs;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / zs;
    const int z = (int)(i - r * zs);
    const float v = z < nz ? what[r * z4 + z] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    qhi[i] = h;
    qlo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// C = (G + lambda I)^-1 (FP64 Cholesky -> FP32) and G + lambda I (FP32), rows padded to z4.
__global__ void __launch_bounds__(128) k_factor_tik(const double* __restrict__ gram, int nz, double lambda,
                                                    float* __restrict__ cinv, float* __restrict__ glam) {
  extern __shared__ double sm[];
  const int ld = nz + 1;
  double* s_a = sm;
  double* s_l = sm + nz * ld;
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

BtLayout make_layout(int nt, int nz, int batch) {
  BtLayout L;
  L.nt = nt;
  L.nz = nz;
  L.z4 = (nz + 3) & ~3;
  L.zs = nz <= 16 ? 16 : (nz <= 32 ? 32 : 64);
  L.tk = (nt + 15) & ~15;
  L.cs = 4 * ((L.z4 / 4) | 1);
  L.batch = batch;
  int off = 0;
  auto take = [&](int bytes) {
    const int at = off;
    off += (bytes + 127) & ~127;
    return at;
  };
  L.off_qh = take(L.tk * L.zs * 2);
  L.off_ql = take(L.tk * L.zs * 2);
  L.off_mh = take(NB * L.tk * 2);
  L.off_ml = take(NB * L.tk * 2);
  L.off_c = take(nz * L.cs * 4);
  L.off_g = take(nz * L.cs * 4);
  L.off_b0 = take(L.zs * NB * 4);
  L.off_bf = take(L.zs * NB * 4);
  L.off_x = take(L.zs * NB * 4);
  L.total = off;
  return L;
}

}  // namespace

size_t batch_tikhonov_smem_bytes(int nt, int nz) { return (size_t)make_layout(nt, nz, 1).total; }

// Build (once per handle) the BF16 tables and (per lambda) C and G + lambda I.
ctof_status batch_tikhonov_prepare(ctof_kernel_s* k, double lambda, cudaStream_t st) {
  const int zs = k->nz <= 16 ? 16 : (k->nz <= 32 ? 32 : 64);
  if (!k->d_qhi) {
    const size_t n = (size_t)k->nclass * k->nt * zs;
    void* p = nullptr;
    if (cudaMalloc(&p, 2 * n * sizeof(__nv_bfloat16)) != cudaSuccess) {
      cudaGetLastError();
      return CTOF_ENOMEM;
    }
    k->d_qhi = p;
    k->d_qlo = static_cast<__nv_bfloat16*>(p) + n;
    k_split_bf16<<<152 * 8, 256, 0, st>>>(k->d_what, (long long)k->nclass * k->nt, k->nz, k->z4, zs,
                                          static_cast<__nv_bfloat16*>(k->d_qhi),
                                          static_cast<__nv_bfloat16*>(k->d_qlo));
    CTOF_CUDA_TRY(cudaGetLastError());
  }
  if (!k->d_bt_cinv) {
    void* p = nullptr;
    if (cudaMalloc(&p, 2 * (size_t)k->nclass * k->nz * k->z4 * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return CTOF_ENOMEM;
    }
    k->d_bt_cinv = static_cast<float*>(p);
    k->d_bt_glam = k->d_bt_cinv + (size_t)k->nclass * k->nz * k->z4;
    k->bt_lambda = -1.0;
  }
  if (k->bt_lambda != lambda) {
    const size_t fsm = (size_t)2 * k->nz * (k->nz + 1) * sizeof(double);
    CTOF_CUDA_TRY(cudaFuncSetAttribute(k_factor_tik, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm));
    k_factor_tik<<<k->nclass, 128, fsm, st>>>(k->d_gram, k->nz, lambda, k->d_bt_cinv, k->d_bt_glam);
    CTOF_CUDA_TRY(cudaGetLastError());
    k->bt_lambda = lambda;
  }
  return CTOF_OK;
}

ctof_status batch_tikhonov_contract(const ctof_kernel_s* k, int batch, const float2* m_hat, int ldm, float2* x_hat,
                                    int ldx, int refine, cudaStream_t st) {
  const BtLayout L = make_layout(k->nt, k->nz, batch);
  if ((size_t)L.total > 227 * 1024) return CTOF_EUNSUPPORTED;
  CTOF_CUDA_TRY(cudaFuncSetAttribute(k_batch_tikhonov_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total));
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, k->device);
  const int grid = k->nclass < nsm ? k->nclass : nsm;
  k_batch_tikhonov_bf16<<<grid, BT_THREADS, L.total, st>>>(
      L, static_cast<const __nv_bfloat16*>(k->d_qhi), static_cast<const __nv_bfloat16*>(k->d_qlo), k->d_bt_cinv,
      k->d_bt_glam, k->d_members, k->nclass, m_hat, ldm, x_hat, ldx, refine);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}
