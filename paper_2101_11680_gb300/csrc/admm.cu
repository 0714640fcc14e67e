// Spatial-domain steps of the ADMM iteration (nonnegativity + anisotropic 3-D
// TV, scaled form).  With a2 = D x + u2 and a3 = x + u3:
//   v2 = soft(a2, beta/rho),  u2 <- a2 - v2,  w2 = v2 - u2 = 2 v2 - a2
//   v3 = max(a3, 0) on the scan support S (0 off S),  u3 <- a3 - v3,  w3 = 2 v3 - a3
//   s  = D^T w2 + w3      (the Z-side part of the next x-update right-hand side)
// D: forward differences, lateral periodic on the P x P grid, axial Neumann
// (Z-1 differences).  One CTA owns a 32 x 8 lateral tile of four depth planes;
// the backward differences of D^T need w2 of the left/upper/previous-plane
// neighbours, which are recomputed from the previous u2 (hence u2 is double
// buffered: blocks read the old copy, write the new one).
#include <cuda_runtime.h>

#include "ctof_internal.h"

namespace {

constexpr int TX = 32, TY = 8;

__device__ __forceinline__ float soft(float a, float thr) {
  const float m = fabsf(a) - thr;
  return m > 0.f ? copysignf(m, a) : 0.f;
}

// One CTA per (32 x 8 lateral tile, ZP consecutive depth planes j0 ..); each
// thread handles its (x, y) in all ZP planes at once: every load of the block
// is issued before the first use, and the axial neighbours of planes inside
// the group come from the staged tiles and registers.  The axial backward
// difference of plane j0 needs w2z of plane j0 - 1, which is pointwise in
// (x[j0-1], x[j0], u2z[j0-1]) and is recomputed here.
constexpr int ZP = 4;

__global__ void __launch_bounds__(TX* TY) k_tv_stencil(const float* __restrict__ x, const float* __restrict__ u2o,
                                                       float* __restrict__ u2n, float* __restrict__ u3,
                                                       float* __restrict__ s_out, const double* __restrict__ beta,
                                                       float inv_rho, int P, int nz, int n,
                                                       float* __restrict__ out_crop) {
  __shared__ float sX[ZP][TY + 2][TX + 2];
  __shared__ float sW2x[ZP][TY][TX + 1];
  __shared__ float sW2y[ZP][TY + 1][TX];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, j0 = blockIdx.z * ZP;
  const int gx = x0 + tx, gy = y0 + ty;
  const size_t plane = (size_t)P * P;
  const float thr = (float)(beta[0]) * inv_rho;
  const bool in_s = gx < n && gy < n;
  const int tid = ty * TX + tx;
  const float* u2oy = u2o + plane * nz;
  const float* u2oz = u2o + 2 * plane * nz;
  const int xl = (gx - 1 + P) & (P - 1), yu = (gy - 1 + P) & (P - 1);
  for (int i = tid; i < ZP * (TY + 2) * (TX + 2); i += TX * TY) {
    const int q = i / ((TY + 2) * (TX + 2)), r = i - q * ((TY + 2) * (TX + 2));
    const int ly = r / (TX + 2), lx = r - ly * (TX + 2);
    const int yy = (y0 + ly - 1 + P) & (P - 1), xx = (x0 + lx - 1 + P) & (P - 1);
    if (j0 + q < nz) sX[q][ly][lx] = x[(size_t)(j0 + q) * plane + (size_t)yy * P + xx];
  }
  const float* base = x + (size_t)gy * P + gx;
  const size_t pix = (size_t)gy * P + gx;
  float vu2x[ZP], vu2y[ZP], vu2z[ZP], vu3[ZP], vlx[ZP], vuy[ZP];
#pragma unroll
  for (int q = 0; q < ZP; ++q) {
    vu2x[q] = vu2y[q] = vu2z[q] = vu3[q] = vlx[q] = vuy[q] = 0.f;
    if (j0 + q < nz) {
      const size_t jp = (size_t)(j0 + q) * plane;
      vu2x[q] = u2o[jp + pix];
      vu2y[q] = u2oy[jp + pix];
      vu2z[q] = u2oz[jp + pix];
      vu3[q] = u3[jp + pix];
      if (tx == 0) vlx[q] = u2o[jp + (size_t)gy * P + xl];
      if (ty == 0) vuy[q] = u2oy[jp + (size_t)yu * P + gx];
    }
  }
  // axial neighbours outside the group: x[j0 - 1], u2z[j0 - 1] and x[j0 + ZP]
  const float xm = j0 > 0 ? base[(size_t)(j0 - 1) * plane] : 0.f;
  const float u2zm = j0 > 0 ? u2oz[(size_t)(j0 - 1) * plane + pix] : 0.f;
  const float xp = j0 + ZP < nz ? base[(size_t)(j0 + ZP) * plane] : 0.f;
  __syncthreads();
  float w2z_prev = 0.f;
  if (j0 > 0) {
    const float a = (sX[0][ty + 1][tx + 1] - xm) + u2zm;
    w2z_prev = 2.f * soft(a, thr) - a;
  }
  float vs[ZP], vv3[ZP];
#pragma unroll
  for (int q = 0; q < ZP; ++q) {
    const int j = j0 + q;
    vs[q] = vv3[q] = 0.f;
    if (j >= nz) continue;
    const size_t idx = (size_t)j * plane + pix;
    const float c = sX[q][ty + 1][tx + 1];
    float w2x, w2y, w2z;
    {
      const float a = (sX[q][ty + 1][tx + 2] - c) + vu2x[q];
      const float v = soft(a, thr);
      u2n[idx] = a - v;
      w2x = 2.f * v - a;
    }
    {
      const float a = (sX[q][ty + 2][tx + 1] - c) + vu2y[q];
      const float v = soft(a, thr);
      u2n[plane * nz + idx] = a - v;
      w2y = 2.f * v - a;
    }
    if (j < nz - 1) {
      const float xn = q + 1 < ZP ? sX[q + 1 < ZP ? q + 1 : 0][ty + 1][tx + 1] : xp;
      const float a = (xn - c) + vu2z[q];
      const float v = soft(a, thr);
      u2n[2 * plane * nz + idx] = a - v;
      w2z = 2.f * v - a;
    } else {
      u2n[2 * plane * nz + idx] = 0.f;
      w2z = 0.f;
    }
    const float a3 = c + vu3[q];
    const float v3 = in_s ? fmaxf(a3, 0.f) : 0.f;
    u3[idx] = a3 - v3;
    vv3[q] = v3;
    sW2x[q][ty][tx + 1] = w2x;
    sW2y[q][ty + 1][tx] = w2y;
    if (tx == 0) {
      const float a = (c - sX[q][ty + 1][0]) + vlx[q];
      sW2x[q][ty][0] = 2.f * soft(a, thr) - a;
    }
    if (ty == 0) {
      const float a = (c - sX[q][0][tx + 1]) + vuy[q];
      sW2y[q][0][tx] = 2.f * soft(a, thr) - a;
    }
    vs[q] = (w2z_prev - w2z) + (2.f * v3 - a3);
    w2z_prev = w2z;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < ZP; ++q) {
    const int j = j0 + q;
    if (j >= nz) continue;
    const size_t idx = (size_t)j * plane + pix;
    s_out[idx] = (sW2x[q][ty][tx] - sW2x[q][ty][tx + 1]) + (sW2y[q][ty][tx] - sW2y[q][ty + 1][tx]) + vs[q];
    if (out_crop && in_s) out_crop[((size_t)j * n + gy) * n + gx] = vv3[q];
  }
}

__global__ void k_max_abs(const float* __restrict__ v, size_t count, unsigned int* __restrict__ out) {
  float mx = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    mx = fmaxf(mx, fabsf(v[i]));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(mx));
}

__global__ void k_set_beta(double* scalars, double beta_fixed, double beta_rel, double inv_s2) {
  if (threadIdx.x == 0) {
    const unsigned int bits = reinterpret_cast<const unsigned int*>(scalars + 1)[0];
    const double mx = (double)__uint_as_float(bits);
    scalars[0] = beta_fixed >= 0.0 ? beta_fixed : beta_rel * mx * inv_s2;
  }
}

__global__ void k_check_finite(const float* __restrict__ v, size_t count, int* __restrict__ flag) {
  int bad = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(v[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// ---- FISTA for the layer-weighted L1 problem (Eq. 8, Eq. 10) ----

// lam[z] = lam0 * sigma(z) / max_z sigma(z), sigma(z) = sqrt(G_zz) of the class
// holding the DC frequency (f = 0), lam0 = scalars[0].  One block.
__global__ void k_fista_lambda(const double* __restrict__ scalars, const double* __restrict__ gram,
                               const int* __restrict__ members, int nclass, int nz, float* __restrict__ lam) {
  __shared__ int s_c;
  __shared__ double s_max;
  if (threadIdx.x == 0) s_c = -1;
  __syncthreads();
  for (int i = threadIdx.x; i < nclass * 4; i += blockDim.x)
    if (members[i] == 0) s_c = i / 4;  // exactly one entry holds frequency 0
  __syncthreads();
  const int c = s_c;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    if (c >= 0)
      for (int z = 0; z < nz; ++z) mx = fmax(mx, sqrt(gram[((size_t)c * nz + z) * nz + z]));
    s_max = mx;
  }
  __syncthreads();
  const double lam0 = scalars[0];
  for (int z = threadIdx.x; z < nz; z += blockDim.x)
    lam[z] = (c >= 0 && s_max > 0.0) ? (float)(lam0 * sqrt(gram[((size_t)c * nz + z) * nz + z]) / s_max)
                                     : (float)lam0;
}

// r -= m
__global__ void k_sub_meas(float* __restrict__ r, const float* __restrict__ m, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    r[i] -= m[i];
}

// One FISTA step per voxel (g = A^T (A y - m) unnormalised; x holds x_{k-1} on entry):
//   x_k = soft(y - g / s^2, lam[z]);  y <- x_k + beta (x_k - x_{k-1});  x <- x_k
__global__ void k_fista_step(float* __restrict__ y, const float* __restrict__ g, float* __restrict__ x,
                             const float* __restrict__ lam, float beta, float inv_s2, int plane, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const float v = y[i] - inv_s2 * g[i];
    const float xn = soft(v, lam[i / plane]);
    const float xo = x[i];
    x[i] = xn;
    y[i] = xn + beta * (xn - xo);
  }
}

// ---- source multiplexing (Section 5, Eq. 12) ----

// In place: every 8 x 8 block of scan points of every plane ([plane][n][n])
// <- H_64 (Sylvester Hadamard) times its 64 values taken row-major.  One warp
// per block, lane l holding entries l and l + 32; the fast Walsh-Hadamard
// butterflies (a + b, a - b) run over strides 1..16 across lanes and 32 in
// registers, which is H_64 in its natural (Sylvester) order.
__global__ void k_block_hadamard(float* __restrict__ v, int planes, int n) {
  const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  const int nb = n >> 3;
  const long long nblk = (long long)planes * nb * nb;
  if (warp >= nblk) return;
  const int plane = (int)(warp / ((long long)nb * nb));
  const int rem = (int)(warp - (long long)plane * nb * nb);
  const int by = rem / nb, bx = rem - by * nb;
  float* base = v + (size_t)plane * n * n + (size_t)(by * 8) * n + bx * 8;
  // entry i -> row i / 8, column i % 8 of the block
  float a = base[(lane >> 3) * n + (lane & 7)];
  float b = base[((lane + 32) >> 3) * n + (lane & 7)];
#pragma unroll
  for (int h = 1; h < 32; h <<= 1) {
    const float pa = __shfl_xor_sync(0xffffffffu, a, h);
    const float pb = __shfl_xor_sync(0xffffffffu, b, h);
    const bool hi = (lane & h) != 0;
    a = hi ? pa - a : a + pa;
    b = hi ? pb - b : b + pb;
  }
  const float s = a + b, d = a - b;
  base[(lane >> 3) * n + (lane & 7)] = s;
  base[((lane + 32) >> 3) * n + (lane & 7)] = d;
}

int grid_elem(size_t count) {
  size_t b = (count + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

ctof_status admm_tv_stencil(const ctof_kernel_s* k, const float* x, const float* u2_old, float* u2_new, float* u3,
                            float* s, const double* beta_dev, float rho, float* out_crop, cudaStream_t st) {
  dim3 block(TX, TY);
  dim3 grid(k->p / TX, k->p / TY, ctof_div_up(k->nz, ZP));
  k_tv_stencil<<<grid, block, 0, st>>>(x, u2_old, u2_new, u3, s, beta_dev, 1.0f / rho, k->p, k->nz, k->n, out_crop);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

// *out_dev (the second device scalar slot) receives max |v| as float bits; the
// slot must be zeroed beforehand.
ctof_status reduce_max_abs(const float* v, size_t count, double* out_dev, cudaStream_t st) {
  int blocks = (int)((count + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  k_max_abs<<<blocks, 256, 0, st>>>(v, count, reinterpret_cast<unsigned int*>(out_dev));
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status admm_set_beta(double* scalars, double beta_fixed, double beta_rel, double inv_scale2, cudaStream_t st) {
  k_set_beta<<<1, 32, 0, st>>>(scalars, beta_fixed, beta_rel, inv_scale2);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status check_finite(const float* v, size_t count, int* flag_dev, cudaStream_t st) {
  int blocks = (int)((count + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  k_check_finite<<<blocks, 256, 0, st>>>(v, count, flag_dev);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status fista_lambda(const ctof_kernel_s* k, const double* scalars, float* lam, cudaStream_t st) {
  k_fista_lambda<<<1, 128, 0, st>>>(scalars, k->d_gram, k->d_members, k->nclass, k->nz, lam);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status fista_sub_meas(float* r, const float* m, size_t count, cudaStream_t st) {
  k_sub_meas<<<grid_elem(count), 256, 0, st>>>(r, m, count);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status fista_step(float* y, const float* g, float* x, const float* lam, float beta, float inv_s2, int plane,
                       size_t count, cudaStream_t st) {
  k_fista_step<<<grid_elem(count), 256, 0, st>>>(y, g, x, lam, beta, inv_s2, plane, count);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status block_hadamard(float* v, int planes, int n, cudaStream_t st) {
  if (n % 8 != 0) return CTOF_EUNSUPPORTED;
  const long long warps = (long long)planes * (n / 8) * (n / 8);
  const long long blocks = (warps * 32 + 255) / 256;
  k_block_hadamard<<<(unsigned)blocks, 256, 0, st>>>(v, planes, n);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}
