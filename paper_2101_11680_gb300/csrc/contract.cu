// Per-frequency contractions of the convolutional model (Eq. 11 in the
// lateral Fourier domain): for every half-plane frequency f,
//   forward  M_hat(f, t) = sum_z W_hat(f, t, z) mu_hat(f, z)       (T x Z . Z)
//   adjoint  V_hat(f, z) = sum_t W_hat(f, t, z) r_hat(f, t)        (Z x T . T)
// W_hat is real (the kernel is even in x and y) and, for dx == dy, equal on
// the up-to-four frequencies (a,b), (a,-b), (b,a), (b,-a) of one class; a CTA
// stages one class's T x Z matrix once in shared memory and applies it to the
// complex vectors of all members (up to 8 real right-hand sides).
// (The fused ADMM x-update lives in contract_admm.cu.)
#include <cuda_runtime.h>

#include "ctof_internal.h"

namespace {

constexpr int CT_THREADS = 256;
constexpr int CT_WARPS = CT_THREADS / 32;

// W_hat is stored [class][nt][z4] (rows padded to a multiple of 4 floats).
__device__ __forceinline__ void load_what(float* s_w, const float* __restrict__ what, int c, int nt, int nz) {
  const int z4 = (nz + 3) & ~3;
  const float* src = what + (size_t)c * nt * z4;
  const int total = nt * nz;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int t = i / nz, z = i - t * nz;
    s_w[t * (nz + 1) + z] = src[(size_t)t * z4 + z];
  }
}

// Partial adjoint sums: warp w covers t in its chunk; lane covers z = lane, lane+32.
__device__ __forceinline__ void adj_partials(const float* s_w, const float2* s_vin, int nt, int nz, int nmem,
                                             float2* s_part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int chunk = (nt + CT_WARPS - 1) / CT_WARPS;
  const int t0 = warp * chunk, t1 = min(nt, t0 + chunk);
  float2 acc0[4], acc1[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) acc0[m] = acc1[m] = make_float2(0.f, 0.f);
  const int z0 = lane, z1 = lane + 32;
  for (int t = t0; t < t1; ++t) {
    const float w0 = z0 < nz ? s_w[t * (nz + 1) + z0] : 0.f;
    const float w1 = z1 < nz ? s_w[t * (nz + 1) + z1] : 0.f;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      if (m < nmem) {
        const float2 v = s_vin[m * nt + t];
        acc0[m].x += w0 * v.x;
        acc0[m].y += w0 * v.y;
        acc1[m].x += w1 * v.x;
        acc1[m].y += w1 * v.y;
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    if (m < nmem) {
      if (z0 < nz) s_part[(warp * 4 + m) * nz + z0] = acc0[m];
      if (z1 < nz) s_part[(warp * 4 + m) * nz + z1] = acc1[m];
    }
  }
}

__device__ __forceinline__ int load_members(const int* __restrict__ members, int c, int (&mem)[4]) {
  int nmem = 0;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    mem[m] = members[c * 4 + m];
    nmem += mem[m] >= 0;
  }
  return nmem;  // members are packed first
}

__global__ void __launch_bounds__(CT_THREADS) k_contract_fwd(const float* __restrict__ what,
                                                             const int* __restrict__ members, int nclass, int nt,
                                                             int nz, const float2* __restrict__ in_z, int ldz,
                                                             float2* __restrict__ out_t, int ldt) {
  extern __shared__ float smem_f[];
  float* s_w = smem_f;
  float2* s_x = reinterpret_cast<float2*>(s_w + ((nt * (nz + 1) + 1) & ~1));
  for (int c = blockIdx.x; c < nclass; c += gridDim.x) {
    int mem[4];
    const int nmem = load_members(members, c, mem);
    load_what(s_w, what, c, nt, nz);
    for (int i = threadIdx.x; i < 4 * nz; i += blockDim.x) {
      const int m = i / nz, z = i - m * nz;
      s_x[i] = m < nmem ? in_z[(size_t)mem[m] * ldz + z] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
      float2 acc[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[m] = make_float2(0.f, 0.f);
      const float* wr = s_w + t * (nz + 1);
      for (int z = 0; z < nz; ++z) {
        const float w = wr[z];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const float2 x = s_x[m * nz + z];
          acc[m].x += w * x.x;
          acc[m].y += w * x.y;
        }
      }
#pragma unroll
      for (int m = 0; m < 4; ++m)
        if (m < nmem) out_t[(size_t)mem[m] * ldt + t] = acc[m];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(CT_THREADS) k_contract_adj(const float* __restrict__ what,
                                                             const int* __restrict__ members, int nclass, int nt,
                                                             int nz, const float2* __restrict__ in_t, int ldt,
                                                             float2* __restrict__ out_z, int ldz) {
  extern __shared__ float smem_f[];
  float* s_w = smem_f;
  float2* s_v = reinterpret_cast<float2*>(s_w + ((nt * (nz + 1) + 1) & ~1));
  float2* s_part = s_v + 4 * nt;
  for (int c = blockIdx.x; c < nclass; c += gridDim.x) {
    int mem[4];
    const int nmem = load_members(members, c, mem);
    load_what(s_w, what, c, nt, nz);
    for (int i = threadIdx.x; i < 4 * nt; i += blockDim.x) {
      const int m = i / nt, t = i - m * nt;
      s_v[i] = m < nmem ? in_t[(size_t)mem[m] * ldt + t] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    adj_partials(s_w, s_v, nt, nz, nmem, s_part);
    __syncthreads();
    for (int i = threadIdx.x; i < nmem * nz; i += blockDim.x) {
      const int m = i / nz, z = i - m * nz;
      float2 acc = make_float2(0.f, 0.f);
      for (int w = 0; w < CT_WARPS; ++w) acc = cadd(acc, s_part[(w * 4 + m) * nz + z]);
      out_z[(size_t)mem[m] * ldz + z] = acc;
    }
    __syncthreads();
  }
}

// Tikhonov: x_hat = (G + lambda I)^-1 W_hat^T m_hat per member, with the FP64
// Cholesky factor L (lower, row-major [nz][nz]) of G + lambda I.
__global__ void __launch_bounds__(CT_THREADS) k_contract_tikhonov(
    const float* __restrict__ what, const double* __restrict__ chol, const int* __restrict__ members, int nclass,
    int nt, int nz, const float2* __restrict__ m_hat, int ldt, float2* __restrict__ x_hat, int ldz) {
  extern __shared__ float smem_f[];
  float* s_w = smem_f;
  float2* s_v = reinterpret_cast<float2*>(s_w + ((nt * (nz + 1) + 1) & ~1));
  float2* s_part = s_v + 4 * nt;
  double* s_l = reinterpret_cast<double*>(s_part + CT_WARPS * 4 * nz);  // [nz][nz]
  double* s_b = s_l + nz * nz;                                         // [4][2][nz]
  for (int c = blockIdx.x; c < nclass; c += gridDim.x) {
    int mem[4];
    const int nmem = load_members(members, c, mem);
    load_what(s_w, what, c, nt, nz);
    for (int i = threadIdx.x; i < nz * nz; i += blockDim.x) s_l[i] = chol[(size_t)c * nz * nz + i];
    for (int i = threadIdx.x; i < 4 * nt; i += blockDim.x) {
      const int m = i / nt, t = i - m * nt;
      s_v[i] = m < nmem ? m_hat[(size_t)mem[m] * ldt + t] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    adj_partials(s_w, s_v, nt, nz, nmem, s_part);
    __syncthreads();
    for (int i = threadIdx.x; i < nmem * nz; i += blockDim.x) {
      const int m = i / nz, z = i - m * nz;
      double ax = 0.0, ay = 0.0;
      for (int w = 0; w < CT_WARPS; ++w) {
        ax += (double)s_part[(w * 4 + m) * nz + z].x;
        ay += (double)s_part[(w * 4 + m) * nz + z].y;
      }
      s_b[(m * 2 + 0) * nz + z] = ax;
      s_b[(m * 2 + 1) * nz + z] = ay;
    }
    __syncthreads();
    // one thread per real right-hand side: L y = b, then L^T x = y
    if (threadIdx.x < 2 * nmem) {
      double* b = s_b + threadIdx.x * nz;
      for (int i = 0; i < nz; ++i) {
        double acc = b[i];
        for (int j = 0; j < i; ++j) acc -= s_l[i * nz + j] * b[j];
        b[i] = acc / s_l[i * nz + i];
      }
      for (int i = nz - 1; i >= 0; --i) {
        double acc = b[i];
        for (int j = i + 1; j < nz; ++j) acc -= s_l[j * nz + i] * b[j];
        b[i] = acc / s_l[i * nz + i];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nmem * nz; i += blockDim.x) {
      const int m = i / nz, z = i - m * nz;
      x_hat[(size_t)mem[m] * ldz + z] =
          make_float2((float)s_b[(m * 2 + 0) * nz + z], (float)s_b[(m * 2 + 1) * nz + z]);
    }
    __syncthreads();
  }
}

size_t what_floats(int nt, int nz) { return (size_t)((nt * (nz + 1) + 1) & ~1); }

int contract_grid(int nclass, size_t smem) {
  int per_sm = (int)(200 * 1024 / (smem + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 8) per_sm = 8;
  int g = 152 * per_sm;
  return nclass < g ? nclass : g;
}

}  // namespace

ctof_status contract_forward(const ctof_kernel_s* k, const float2* in_z, float2* out_t, cudaStream_t st) {
  const size_t sm = what_floats(k->nt, k->nz) * 4 + (size_t)4 * k->nz * 8;
  CTOF_CUDA_TRY(cudaFuncSetAttribute(k_contract_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_contract_fwd<<<contract_grid(k->nclass, sm), CT_THREADS, sm, st>>>(k->d_what, k->d_members, k->nclass, k->nt,
                                                                       k->nz, in_z, k->ldz, out_t, k->ldt);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status contract_adjoint(const ctof_kernel_s* k, const float2* in_t, float2* out_z, cudaStream_t st) {
  const size_t sm = what_floats(k->nt, k->nz) * 4 + (size_t)4 * k->nt * 8 + (size_t)CT_WARPS * 4 * k->nz * 8;
  CTOF_CUDA_TRY(cudaFuncSetAttribute(k_contract_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_contract_adj<<<contract_grid(k->nclass, sm), CT_THREADS, sm, st>>>(k->d_what, k->d_members, k->nclass, k->nt,
                                                                       k->nz, in_t, k->ldt, out_z, k->ldz);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status contract_tikhonov(const ctof_kernel_s* k, const double* chol, const float2* m_hat, float2* x_hat,
                              cudaStream_t st) {
  const int nt = k->nt, nz = k->nz;
  size_t sm = what_floats(nt, nz) * 4 + (size_t)4 * nt * 8 + (size_t)CT_WARPS * 4 * nz * 8;
  sm = (sm + 7) & ~(size_t)7;
  sm += ((size_t)nz * nz + 8 * (size_t)nz) * 8;
  CTOF_CUDA_TRY(cudaFuncSetAttribute(k_contract_tikhonov, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_contract_tikhonov<<<contract_grid(k->nclass, sm), CT_THREADS, sm, st>>>(
      k->d_what, chol, k->d_members, k->nclass, nt, nz, m_hat, k->ldt, x_hat, k->ldz);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}
