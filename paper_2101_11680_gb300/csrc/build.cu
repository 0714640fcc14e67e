// One-time construction of the sensitivity kernel and its per-frequency
// factorisations (Section 3: computing the sensitivity matrix is a one-time
// process).  Everything here runs in FP64 on the device:
//
//  1. W[k][j][|oy|][|ox|] = dx dy dz * int_bin_k (Phi0 (*)_t R)(rho, z_j, t) dt
//     (Eq. 5), the time convolution in closed form from the Laplace
//     transforms of the semi-infinite extrapolated-boundary Green's
//     functions, the bin integral by an 8-node Gauss-Legendre rule on each of
//     4 equal pieces of the bin.  Fluorescence mode (Section 5): Phi0 of the
//     excitation optics, R of the emission optics and a lifetime
//     convolution, through the product of Laplace transforms and a
//     fixed-Talbot inversion at the bin edges (k_w_quadrant_fl).
//  2. W_hat = the 2-D DFT of the periodic kernel.  The kernel is even in x
//     and y, so W_hat is real and is a separable cosine sum over the
//     non-negative offsets: W_hat(a,b) = sum_{q,p} c_q c_p W[q][p]
//     cos(2 pi b q/P) cos(2 pi a p/P) (c = multiplicity of +-offset), done as
//     two batched FP64 GEMMs per (t,z) plane and gathered per frequency class.
//  3. Gram G(f) = W_hat(f)^T W_hat(f) (FP64), the normalisation
//     s = sigma_max(W_hat(0)) (the DC block dominates every other frequency
//     entrywise since W >= 0), and the ADMM normal matrix
//     H = G/s^2 + (|dx|^2 + |dy|^2 + 1) I + Dz^T Dz, Cholesky-factored and
//     inverted in FP64, stored FP32.
#include <cuda_runtime.h>
#include <math.h>

#include <vector>

#include "ctof_internal.h"

namespace {

struct PhysParams {
  double mua, D, c, kappa, zb, z0, rmin;
  double dx, dy, dz, zfirst, dt, vol;
  double gl_x[8], gl_w[8];
};

// Voxel averaging of the first `layers` depth layers: the voxel's weight is the
// integral of the kernel over the voxel (the time-domain forward model
// integrates J mu over the volume, mu constant per voxel), taken with a tensor
// Gauss-Legendre rule of `nodes` points per axis around the voxel centre; the
// other layers keep the centre value (the midpoint rule).
struct AvgParams {
  int layers, nodes;
  double x[8], w[8];  // nodes and weights on [-1, 1]
};

// Bin integral of (Phi0 (*) R)(rho, z, t) over bin kbin (32-node composite rule).
__device__ double abs_point_bin(double rho2, double z, int kbin, const PhysParams& prm) {
  double r[4];
  r[0] = sqrt(rho2 + (z - prm.z0) * (z - prm.z0));
  r[1] = sqrt(rho2 + (z + prm.z0 + 2.0 * prm.zb) * (z + prm.z0 + 2.0 * prm.zb));
  r[2] = sqrt(rho2 + z * z);
  r[3] = sqrt(rho2 + (z + 2.0 * prm.zb) * (z + 2.0 * prm.zb));
#pragma unroll
  for (int i = 0; i < 4; ++i) r[i] = fmax(r[i], prm.rmin);
  // four source/detector image pairs (i in {1,2}, j in {3,4})
  double pre[4], a[4], a2[4], rj[4];
  const double zz[2] = {z, z + 2.0 * prm.zb};
  const double pi = 3.14159265358979323846;
#pragma unroll
  for (int ii = 0; ii < 2; ++ii) {
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      const int e = ii * 2 + jj;
      const double ri = r[ii], rjj = r[2 + jj];
      pre[e] = (ii == 0 ? 1.0 : -1.0) * zz[jj] / (16.0 * pi * pi * prm.D * ri * rjj * rjj * rjj);
      a[e] = ri + rjj;
      a2[e] = a[e] * a[e];
      rj[e] = rjj;
    }
  }
  const double base_c = 1.0 / (2.0 * sqrt(pi * prm.kappa));
  const double hsub = prm.dt * 0.25;
  const double muac = prm.mua * prm.c;
  double acc = 0.0;
  for (int s = 0; s < 4; ++s) {
    const double ta = kbin * prm.dt + s * hsub;
#pragma unroll
    for (int gi = 0; gi < 8; ++gi) {
      const double t = ta + 0.5 * hsub * (prm.gl_x[gi] + 1.0);
      const double inv4 = 1.0 / (4.0 * prm.kappa * t);
      double val = 0.0;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const double arg = -a2[e] * inv4 - muac * t;
        if (arg > -745.0) val += pre[e] * exp(arg) * (a[e] + rj[e] * (2.0 * a2[e] * inv4 - 1.0));
      }
      acc += 0.5 * hsub * prm.gl_w[gi] * base_c * val / (t * sqrt(t));
    }
  }
  return acc;
}

// (qy, qx) of quadrant pair index pr (lower triangle when symmetric, else row-major)
__device__ __forceinline__ void pair_of(long long pr, int q, int symmetric, int& qy, int& qx) {
  if (symmetric) {
    qy = (int)((sqrt(8.0 * (double)pr + 1.0) - 1.0) * 0.5);
    while ((long long)(qy + 1) * (qy + 2) / 2 <= pr) ++qy;
    while ((long long)qy * (qy + 1) / 2 > pr) --qy;
    qx = (int)(pr - (long long)qy * (qy + 1) / 2);
  } else {
    qy = (int)(pr / q);
    qx = (int)(pr - (long long)qy * q);
  }
}

__global__ void k_w_quadrant(double* __restrict__ w, int t0, int tcount, int nz, int q, int symmetric,
                             PhysParams prm, AvgParams av) {
  const long long npairs = symmetric ? (long long)q * (q + 1) / 2 : (long long)q * q;
  const long long total = npairs * nz;
  for (long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x; gid < total;
       gid += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(gid / npairs);
    int qy, qx;
    pair_of(gid - (long long)j * npairs, q, symmetric, qy, qx);
    const double z = prm.zfirst + j * prm.dz;
    const int ns = j < av.layers ? av.nodes : 1;
    for (int tk = 0; tk < tcount; ++tk) {
      const int kbin = t0 + tk;
      double acc = 0.0;
      if (ns == 1) {
        acc = abs_point_bin((qx * prm.dx) * (qx * prm.dx) + (qy * prm.dy) * (qy * prm.dy), z, kbin, prm);
      } else {
        for (int c = 0; c < ns; ++c)
          for (int b = 0; b < ns; ++b)
            for (int a = 0; a < ns; ++a) {
              const double px = qx * prm.dx + 0.5 * prm.dx * av.x[a];
              const double py = qy * prm.dy + 0.5 * prm.dy * av.x[b];
              const double pz = z + 0.5 * prm.dz * av.x[c];
              acc += av.w[a] * av.w[b] * av.w[c] * 0.125 * abs_point_bin(px * px + py * py, pz, kbin, prm);
            }
      }
      acc *= prm.vol;
      w[(((size_t)tk * nz + j) * q + qy) * q + qx] = acc;
      if (symmetric && qx != qy) w[(((size_t)tk * nz + j) * q + qx) * q + qy] = acc;
    }
  }
}

// ---- fluorescence mode ----
// f = Phi0_ex (*)_t L_tau (*)_t R_em.  Its Laplace transform is the product of
// the three factors' closed-form transforms (q = sqrt((s + mua c)/(D c)) of
// each medium):
//   F(s) = [e^{-r1 q_ex}/r1 - e^{-r2 q_ex}/r2] / (4 pi D_ex)
//        * [z (1 + r3 q_em) e^{-r3 q_em}/r3^3 + (z + 2 zb_em)(1 + r4 q_em) e^{-r4 q_em}/r4^3] / (4 pi)
//        / (1 + s tau).
// The cumulative response C(t) = int_0^t f is the inverse transform of F(s)/s,
// taken with the fixed-Talbot rule (Abate and Valko 2004): on the contour
// s(theta) = r theta (cot theta + i), r = 2M/(5t), the trapezoidal rule in
// theta gives C(t) = (r/M) sum_j Re(gamma_j G(r u_j)) with u_j = theta_j
// cot theta_j + i theta_j (u_0 = 1) and weights gamma_j = e^{(2M/5) u_j}
// (1 + i sigma_j), sigma = theta + (theta cot theta - 1) cot theta,
// gamma_0 = e^{2M/5}/2; since t r = 2M/5 the weights do not depend on t.
// The bin integral is C at the upper edge minus C at the lower edge.
constexpr int TALBOT_M = 24;

struct FluoParams {
  double a_ex, k_ex, D_ex, zb_ex, z0;  // a = mua c, k = D c
  double a_em, k_em, zb_em;
  double tau, rmin, dx, dy, dz, zfirst, dt, vol;
  double u_re[TALBOT_M], u_im[TALBOT_M];
  double g_re[TALBOT_M], g_im[TALBOT_M];
};

struct cd {
  double re, im;
};
__device__ __forceinline__ cd c_mul(cd a, cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cd c_div(cd a, cd b) {
  // Smith's algorithm
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, d = b.re + b.im * r;
    return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
  }
  const double r = b.re / b.im, d = b.re * r + b.im;
  return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}
// principal square root, written to avoid cancellation in either half-plane
__device__ __forceinline__ cd c_sqrt(cd a) {
  const double m = hypot(a.re, a.im);
  if (m == 0.0) return {0.0, 0.0};
  if (a.re >= 0.0) {
    const double t = sqrt(0.5 * (m + a.re));
    return {t, a.im / (2.0 * t)};
  }
  const double t = sqrt(0.5 * (m - a.re));
  return {fabs(a.im) / (2.0 * t), copysign(t, a.im)};
}
// e^{-x a}, x >= 0 and Re a >= 0 (no overflow)
__device__ __forceinline__ cd c_exp_neg(double x, cd a) {
  const double e = exp(-x * a.re);
  double sn, cs;
  sincos(x * a.im, &sn, &cs);
  return {e * cs, -e * sn};
}

__device__ double fl_cumulative_at(double t, double rho2, double z, const FluoParams& p) {
  const double pi = 3.14159265358979323846;
  const double r1 = fmax(sqrt(rho2 + (z - p.z0) * (z - p.z0)), p.rmin);
  const double r2 = fmax(sqrt(rho2 + (z + p.z0 + 2.0 * p.zb_ex) * (z + p.z0 + 2.0 * p.zb_ex)), p.rmin);
  const double r3 = fmax(sqrt(rho2 + z * z), p.rmin);
  const double r4 = fmax(sqrt(rho2 + (z + 2.0 * p.zb_em) * (z + 2.0 * p.zb_em)), p.rmin);
  const double r = 2.0 * TALBOT_M / (5.0 * t);
  const double z4 = z + 2.0 * p.zb_em;
  double acc = 0.0;
  for (int j = 0; j < TALBOT_M; ++j) {
    const cd s = {r * p.u_re[j], r * p.u_im[j]};
    const cd qx = c_sqrt({(s.re + p.a_ex) / p.k_ex, s.im / p.k_ex});
    const cd qm = c_sqrt({(s.re + p.a_em) / p.k_em, s.im / p.k_em});
    const cd e1 = c_exp_neg(r1, qx), e2 = c_exp_neg(r2, qx);
    const cd src = {(e1.re / r1 - e2.re / r2) / (4.0 * pi * p.D_ex), (e1.im / r1 - e2.im / r2) / (4.0 * pi * p.D_ex)};
    const cd e3 = c_exp_neg(r3, qm), e4 = c_exp_neg(r4, qm);
    const cd f3 = c_mul({1.0 + r3 * qm.re, r3 * qm.im}, e3);
    const cd f4 = c_mul({1.0 + r4 * qm.re, r4 * qm.im}, e4);
    const double w3 = z / (4.0 * pi * r3 * r3 * r3), w4 = z4 / (4.0 * pi * r4 * r4 * r4);
    const cd det = {w3 * f3.re + w4 * f4.re, w3 * f3.im + w4 * f4.im};
    // G(s) = src det / ((1 + s tau) s)
    const cd den = c_mul({1.0 + s.re * p.tau, s.im * p.tau}, s);
    const cd g = c_div(c_mul(src, det), den);
    acc += p.g_re[j] * g.re - p.g_im[j] * g.im;
  }
  return r / TALBOT_M * acc;
}

// Cumulative response at time t, voxel-averaged when ns > 1 (the average of
// the cumulative is the cumulative of the average).
__device__ double fl_cumulative(double t, int qx, int qy, double z, int ns, const FluoParams& p, const AvgParams& av) {
  if (ns == 1) return fl_cumulative_at(t, (qx * p.dx) * (qx * p.dx) + (qy * p.dy) * (qy * p.dy), z, p);
  double acc = 0.0;
  for (int c = 0; c < ns; ++c)
    for (int b = 0; b < ns; ++b)
      for (int a = 0; a < ns; ++a) {
        const double px = qx * p.dx + 0.5 * p.dx * av.x[a];
        const double py = qy * p.dy + 0.5 * p.dy * av.x[b];
        const double pz = z + 0.5 * p.dz * av.x[c];
        acc += av.w[a] * av.w[b] * av.w[c] * 0.125 * fl_cumulative_at(t, px * px + py * py, pz, p);
      }
  return acc;
}

__global__ void k_w_quadrant_fl(double* __restrict__ w, int t0, int tcount, int nz, int q, int symmetric,
                                FluoParams prm, AvgParams av) {
  const long long npairs = symmetric ? (long long)q * (q + 1) / 2 : (long long)q * q;
  const long long total = npairs * nz;
  for (long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x; gid < total;
       gid += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(gid / npairs);
    int qy, qx;
    pair_of(gid - (long long)j * npairs, q, symmetric, qy, qx);
    const double z = prm.zfirst + j * prm.dz;
    const int ns = j < av.layers ? av.nodes : 1;
    double prev = t0 > 0 ? fl_cumulative(t0 * prm.dt, qx, qy, z, ns, prm, av) : 0.0;
    for (int tk = 0; tk < tcount; ++tk) {
      const double cur = fl_cumulative((t0 + tk + 1) * prm.dt, qx, qy, z, ns, prm, av);
      const double acc = (cur - prev) * prm.vol;
      prev = cur;
      w[(((size_t)tk * nz + j) * q + qy) * q + qx] = acc;
      if (symmetric && qx != qy) w[(((size_t)tk * nz + j) * q + qx) * q + qy] = acc;
    }
  }
}

void make_fluo_params(const ctof_kernel_s* k, FluoParams& p) {
  const double n = k->optics.n;
  const double c = 0.299792458 / n;
  const double reff = -1.440 / (n * n) + 0.710 / n + 0.668 + 0.0636 * n;
  const double Acoef = (1.0 + reff) / (1.0 - reff);
  const double mx = k->optics.mua_mm, sx = k->optics.musp_mm;
  const double mm = k->emission.mua_mm, sm = k->emission.musp_mm;
  p.D_ex = 1.0 / (3.0 * (mx + sx));
  p.a_ex = mx * c;
  p.k_ex = p.D_ex * c;
  p.zb_ex = 2.0 * Acoef * p.D_ex;
  p.z0 = k->optics.z0_mm > 0 ? k->optics.z0_mm : 1.0 / (mx + sx);
  const double D_em = 1.0 / (3.0 * (mm + sm));
  p.a_em = mm * c;
  p.k_em = D_em * c;
  p.zb_em = 2.0 * Acoef * D_em;
  p.tau = k->emission.tau_ps;
  p.rmin = k->r_min;
  p.dx = k->grid.dx_mm;
  p.dy = k->grid.dy_mm;
  p.dz = k->grid.dz_mm;
  p.zfirst = k->grid.z_first_mm;
  p.dt = k->grid.dt_ps;
  p.vol = p.dx * p.dy * p.dz;
  const double pi = 3.14159265358979323846;
  const double cm = 2.0 * TALBOT_M / 5.0;
  p.u_re[0] = 1.0;
  p.u_im[0] = 0.0;
  p.g_re[0] = 0.5 * exp(cm);
  p.g_im[0] = 0.0;
  for (int j = 1; j < TALBOT_M; ++j) {
    const double th = j * pi / TALBOT_M;
    const double cot = cos(th) / sin(th);
    const double sigma = th + (th * cot - 1.0) * cot;
    p.u_re[j] = th * cot;
    p.u_im[j] = th;
    const double e = exp(cm * th * cot);
    const double er = e * cos(cm * th), ei = e * sin(cm * th);
    p.g_re[j] = er - ei * sigma;  // e^{cm u} (1 + i sigma)
    p.g_im[j] = ei + er * sigma;
  }
}

// Batched row-major FP64 GEMM C[b] = A[b] * B[b] (M x K times K x N), strides
// per batch (0 = shared operand).  64 x 64 tile, 256 threads, 4 x 4 per thread.
__global__ void __launch_bounds__(256) k_dgemm(const double* __restrict__ A, long long sA, int lda,
                                               const double* __restrict__ B, long long sB, int ldb,
                                               double* __restrict__ C, long long sC, int ldc, int M, int N,
                                               int K) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const int bz = blockIdx.z;
  const double* a = A + bz * sA;
  const double* b = B + bz * sB;
  double* cmat = C + bz * sC;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int i = threadIdx.x; i < 16 * 64; i += 256) {
      const int kk = i & 15, mm = i >> 4;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? a[(size_t)gm * lda + gk] : 0.0;
      const int nn = i & 63, kb = i >> 6;
      const int gn = n0 + nn, gkb = k0 + kb;
      Bs[kb][nn] = (gn < N && gkb < K) ? b[(size_t)gkb * ldb + gn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn < N) cmat[(size_t)gm * ldc + gn] = acc[i][j];
    }
  }
}

// what64[c][plane0 + pl] = out[pl][b_c][a_c]
__global__ void k_gather_classes(const double* __restrict__ out, int nplanes_chunk, int A,
                                 const int2* __restrict__ ab, int nclass, double* __restrict__ what64,
                                 long long ld_what, int plane0) {
  const long long total = (long long)nplanes_chunk * nclass;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int pl = (int)(i / nclass);
    const int c = (int)(i - (long long)pl * nclass);
    const int2 v = ab[c];
    what64[(size_t)c * ld_what + plane0 + pl] = out[((size_t)pl * A + v.y) * A + v.x];
  }
}

// FP32 copy of W_hat with rows padded to z4 floats: out[c][t][z4] (zero padding).
__global__ void k_to_float_padded(const double* __restrict__ in, float* __restrict__ out, long long rows, int nz,
                                  int z4) {
  const long long n = rows * z4;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / z4;
    const int z = (int)(i - r * z4);
    out[i] = z < nz ? (float)in[r * nz + z] : 0.f;
  }
}

// G[c] = sum_t what64[c][t][:]^T what64[c][t][:]
__global__ void __launch_bounds__(256) k_gram(const double* __restrict__ what64, int nt, int nz,
                                              double* __restrict__ gram) {
  constexpr int TC = 16;
  __shared__ double s[TC * 64];
  const int c = blockIdx.x;
  const double* src = what64 + (size_t)c * nt * nz;
  const int npair = nz * nz;
  double acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.0;
  for (int t0 = 0; t0 < nt; t0 += TC) {
    const int tc = min(TC, nt - t0);
    for (int i = threadIdx.x; i < tc * nz; i += blockDim.x) s[i] = src[(size_t)t0 * nz + i];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int pidx = threadIdx.x + r * 256;
      if (pidx < npair) {
        const int z1 = pidx / nz, z2 = pidx - z1 * nz;
        double v = acc[r];
        for (int t = 0; t < tc; ++t) v = fma(s[t * nz + z1], s[t * nz + z2], v);
        acc[r] = v;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int pidx = threadIdx.x + r * 256;
    if (pidx < npair) gram[(size_t)c * npair + pidx] = acc[r];
  }
}

// Largest eigenvalue of the (symmetric positive semi-definite) DC Gram block
// by power iteration; writes sqrt(lambda_max) to *out.
__global__ void k_power_iteration(const double* __restrict__ g, int nz, int iters, double* __restrict__ out) {
  __shared__ double v[64], w[64], red[64];
  const int z = threadIdx.x;
  if (z < nz) v[z] = 1.0 / sqrt((double)nz);
  __syncthreads();
  double lam = 0.0;
  for (int it = 0; it < iters; ++it) {
    if (z < nz) {
      double acc = 0.0;
      for (int q = 0; q < nz; ++q) acc = fma(g[z * nz + q], v[q], acc);
      w[z] = acc;
      red[z] = acc * acc;
    }
    __syncthreads();
    if (z == 0) {
      double s = 0.0;
      for (int q = 0; q < nz; ++q) s += red[q];
      red[0] = sqrt(s);
    }
    __syncthreads();
    const double nrm = red[0];
    __syncthreads();
    if (z < nz) v[z] = nrm > 0 ? w[z] / nrm : 0.0;
    __syncthreads();
  }
  // Rayleigh quotient v^T G v
  if (z < nz) {
    double acc = 0.0;
    for (int q = 0; q < nz; ++q) acc = fma(g[z * nz + q], v[q], acc);
    red[z] = acc * v[z];
  }
  __syncthreads();
  if (z == 0) {
    for (int q = 0; q < nz; ++q) lam += red[q];
    out[0] = sqrt(fmax(lam, 0.0));
  }
}

__global__ void k_max_diag(const double* __restrict__ gram, int nclass, int nz, double* __restrict__ out) {
  __shared__ double red[256];
  double mx = 0.0;
  for (long long i = threadIdx.x; i < (long long)nclass * nz; i += blockDim.x) {
    const int c = (int)(i / nz), j = (int)(i - (long long)c * nz);
    mx = fmax(mx, gram[((size_t)c * nz + j) * nz + j]);
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// In-place lower Cholesky of the symmetric matrix in s_a ([nz][nz+1]).
__device__ void block_cholesky(double* s_a, int nz) {
  const int ld = nz + 1;
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
}

// mode 0: ADMM  H = G/s^2 + (lap+1) I + Dz^T Dz
// mode 1: Tikhonov  H = G + lambda I
// H^-1 = L^-T L^-1 through the FP64 Cholesky factor (exactly symmetric), stored
// FP32 into out32 [nz][z4].
__global__ void __launch_bounds__(128) k_factor(const double* __restrict__ gram, const float* __restrict__ lap,
                                                int nz, double inv_s2, double lambda, int mode,
                                                float* __restrict__ out32, double* __restrict__ out64) {
  extern __shared__ double sm[];
  const int ld = nz + 1;
  double* s_a = sm;
  double* s_l = sm + nz * ld;
  const int c = blockIdx.x;
  const double* g = gram + (size_t)c * nz * nz;
  for (int idx = threadIdx.x; idx < nz * nz; idx += blockDim.x) {
    const int i = idx / nz, j = idx - i * nz;
    double v;
    if (mode == 0) {
      v = g[idx] * inv_s2;
      if (i == j) v += (double)lap[c] + 1.0 + (i > 0 ? 1.0 : 0.0) + (i < nz - 1 ? 1.0 : 0.0);
      if (j == i + 1 || i == j + 1) v -= 1.0;
    } else {
      v = g[idx] + (i == j ? lambda : 0.0);
    }
    s_a[i * ld + j] = v;
  }
  __syncthreads();
  block_cholesky(s_a, nz);
  // L^-1 column by column (one thread per column), then H^-1 = L^-T L^-1.
  for (int col = threadIdx.x; col < nz; col += blockDim.x) {
    for (int i = 0; i < col; ++i) s_l[i * ld + col] = 0.0;
    for (int i = col; i < nz; ++i) {
      double acc = (i == col) ? 1.0 : 0.0;
      for (int kk = col; kk < i; ++kk) acc -= s_a[i * ld + kk] * s_l[kk * ld + col];
      s_l[i * ld + col] = acc / s_a[i * ld + i];
    }
  }
  __syncthreads();
  const int z4 = (nz + 3) & ~3;
  for (int idx = threadIdx.x; idx < nz * z4; idx += blockDim.x) {
    const int i = idx / z4, j = idx - i * z4;
    double acc = 0.0;
    if (j < nz)
      for (int kk = (i > j ? i : j); kk < nz; ++kk) acc += s_l[kk * ld + i] * s_l[kk * ld + j];
    out32[(size_t)c * nz * z4 + idx] = (float)acc;
  }
}

// Gauss-Legendre nodes/weights on [-1,1] by Newton's method on P_n (the
// three-term recurrence gives P_n and P_n').
void gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes); }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

}  // namespace

ctof_status build_kernel_tables(ctof_kernel_s* k, cudaStream_t st) {
  const int nt = k->nt, nz = k->nz, q = k->q, P = k->p, A = P / 2 + 1;
  const int nclass = k->nclass;

  // ---- host tables: class (a, b) pairs and cosine-sum matrices ----
  std::vector<int> members(nclass * 4);
  CTOF_CUDA_TRY(cudaMemcpy(members.data(), k->d_members, members.size() * sizeof(int), cudaMemcpyDeviceToHost));
  std::vector<int2> ab(nclass);
  for (int c = 0; c < nclass; ++c) {
    const int f = members[c * 4];
    const int kx = f % k->h, ky = f / k->h;
    const int b = ky <= P / 2 ? ky : P - ky;
    ab[c] = make_int2(kx, b);  // W_hat(kx, |ky|): x index kx, y index |ky|
  }
  // multiplicity of each non-negative offset on the periodic grid
  std::vector<double> mult(q);
  for (int o = 0; o < q; ++o) {
    if (k->grid.conv_mode == CTOF_LINEAR) mult[o] = o == 0 ? 1.0 : 2.0;
    else mult[o] = (o == 0 || 2 * o == P) ? 1.0 : 2.0;
  }
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<double> cp((size_t)q * A), cqt((size_t)A * q);
  for (int o = 0; o < q; ++o)
    for (int a = 0; a < A; ++a) {
      const long long ph = ((long long)a * o) % P;
      const double v = mult[o] * cos(two_pi * (double)ph / (double)P);
      cp[(size_t)o * A + a] = v;
      cqt[(size_t)a * q + o] = v;
    }

  PhysParams prm;
  {
    const double n = k->optics.n, mua = k->optics.mua_mm, musp = k->optics.musp_mm;
    prm.mua = mua;
    prm.c = 0.299792458 / n;
    prm.D = 1.0 / (3.0 * (mua + musp));
    prm.kappa = prm.D * prm.c;
    const double reff = -1.440 / (n * n) + 0.710 / n + 0.668 + 0.0636 * n;
    const double Acoef = (1.0 + reff) / (1.0 - reff);
    prm.zb = 2.0 * Acoef * prm.D;
    prm.z0 = k->optics.z0_mm > 0 ? k->optics.z0_mm : 1.0 / (mua + musp);
    prm.rmin = k->r_min;
    prm.dx = k->grid.dx_mm;
    prm.dy = k->grid.dy_mm;
    prm.dz = k->grid.dz_mm;
    prm.zfirst = k->grid.z_first_mm;
    prm.dt = k->grid.dt_ps;
    prm.vol = prm.dx * prm.dy * prm.dz;
    gauss_legendre(8, prm.gl_x, prm.gl_w);
  }
  FluoParams fprm;
  if (k->fluorescence) make_fluo_params(k, fprm);
  AvgParams av;
  av.layers = k->avg.layers;
  av.nodes = k->avg.layers > 0 ? k->avg.nodes : 1;
  for (int i = 0; i < 8; ++i) av.x[i] = av.w[i] = 0.0;
  if (av.nodes > 1) gauss_legendre(av.nodes, av.x, av.w);

  // ---- device temporaries, processed in chunks of time bins ----
  const long long planes = (long long)nt * nz;
  int tchunk = nt;
  const long long max_plane_elems = 1LL << 28;  // ~2 GB of FP64 per temporary
  while (tchunk > 1 && (long long)tchunk * nz * (long long)q * (q > A ? q : A) > max_plane_elems) tchunk = (tchunk + 1) / 2;
  const long long chunk_planes = (long long)tchunk * nz;

  DevBuf d_cp, d_cqt, d_ab, d_wq, d_t1, d_out, d_what64, d_scal;
  CTOF_CUDA_TRY(d_cp.alloc(cp.size() * sizeof(double)));
  CTOF_CUDA_TRY(d_cqt.alloc(cqt.size() * sizeof(double)));
  CTOF_CUDA_TRY(d_ab.alloc(ab.size() * sizeof(int2)));
  CTOF_CUDA_TRY(d_wq.alloc((size_t)chunk_planes * q * q * sizeof(double)));
  CTOF_CUDA_TRY(d_t1.alloc((size_t)chunk_planes * q * A * sizeof(double)));
  CTOF_CUDA_TRY(d_out.alloc((size_t)chunk_planes * A * A * sizeof(double)));
  CTOF_CUDA_TRY(d_what64.alloc((size_t)nclass * planes * sizeof(double)));
  CTOF_CUDA_TRY(d_scal.alloc(4 * sizeof(double)));
  CTOF_CUDA_TRY(cudaMemcpyAsync(d_cp.p, cp.data(), cp.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  CTOF_CUDA_TRY(cudaMemcpyAsync(d_cqt.p, cqt.data(), cqt.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  CTOF_CUDA_TRY(cudaMemcpyAsync(d_ab.p, ab.data(), ab.size() * sizeof(int2), cudaMemcpyHostToDevice, st));

  for (int t0 = 0; t0 < nt; t0 += tchunk) {
    const int tc = (t0 + tchunk <= nt) ? tchunk : nt - t0;
    const long long np = (long long)tc * nz;
    {
      const long long npairs = k->symmetric ? (long long)q * (q + 1) / 2 : (long long)q * q;
      const long long work = npairs * nz;
      int blocks = (int)((work + 127) / 128);
      if (blocks > 152 * 64) blocks = 152 * 64;
      if (k->fluorescence) {
        k_w_quadrant_fl<<<blocks, 128, 0, st>>>(d_wq.as<double>(), t0, tc, nz, q, k->symmetric, fprm, av);
      } else {
        k_w_quadrant<<<blocks, 128, 0, st>>>(d_wq.as<double>(), t0, tc, nz, q, k->symmetric, prm, av);
      }
      CTOF_CUDA_TRY(cudaGetLastError());
    }
    if (k->d_w) {
      CTOF_CUDA_TRY(cudaMemcpyAsync(k->d_w + (size_t)t0 * nz * q * q, d_wq.p, (size_t)np * q * q * sizeof(double),
                                    cudaMemcpyDeviceToDevice, st));
    }
    for (long long b0 = 0; b0 < np; b0 += 65535) {
      const int nb = (int)((np - b0) < 65535 ? (np - b0) : 65535);
      dim3 g1(ctof_div_up(A, 64), ctof_div_up(q, 64), nb);
      k_dgemm<<<g1, 256, 0, st>>>(d_wq.as<double>() + b0 * q * q, (long long)q * q, q, d_cp.as<double>(), 0, A,
                                  d_t1.as<double>() + b0 * q * A, (long long)q * A, A, q, A, q);
      CTOF_CUDA_TRY(cudaGetLastError());
      dim3 g2(ctof_div_up(A, 64), ctof_div_up(A, 64), nb);
      k_dgemm<<<g2, 256, 0, st>>>(d_cqt.as<double>(), 0, q, d_t1.as<double>() + b0 * q * A, (long long)q * A, A,
                                  d_out.as<double>() + b0 * A * A, (long long)A * A, A, A, A, q);
      CTOF_CUDA_TRY(cudaGetLastError());
    }
    {
      const long long work = np * nclass;
      int blocks = (int)((work + 255) / 256);
      if (blocks > 152 * 32) blocks = 152 * 32;
      k_gather_classes<<<blocks, 256, 0, st>>>(d_out.as<double>(), (int)np, A, d_ab.as<int2>(), nclass,
                                               d_what64.as<double>(), planes, (int)((long long)t0 * nz));
      CTOF_CUDA_TRY(cudaGetLastError());
    }
  }
  // FP32 copy of W_hat (layout [c][t][z] == [c][plane])
  k_to_float_padded<<<152 * 8, 256, 0, st>>>(d_what64.as<double>(), k->d_what, (long long)nclass * nt, nz,
                                             k->z4);
  CTOF_CUDA_TRY(cudaGetLastError());
  k_gram<<<nclass, 256, 0, st>>>(d_what64.as<double>(), nt, nz, k->d_gram);
  CTOF_CUDA_TRY(cudaGetLastError());
  // class 0 is the DC frequency
  k_power_iteration<<<1, 64, 0, st>>>(k->d_gram, nz, 4000, d_scal.as<double>());
  CTOF_CUDA_TRY(cudaGetLastError());
  k_max_diag<<<1, 256, 0, st>>>(k->d_gram, nclass, nz, d_scal.as<double>() + 1);
  CTOF_CUDA_TRY(cudaGetLastError());
  double scal[2];
  CTOF_CUDA_TRY(cudaMemcpyAsync(scal, d_scal.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CTOF_CUDA_TRY(cudaStreamSynchronize(st));
  k->scale = scal[0];
  k->gram_max = scal[1];
  if (!(k->scale > 0.0) || !isfinite(k->scale)) return CTOF_ENONFINITE;
  const size_t fsm = (size_t)2 * nz * (nz + 1) * sizeof(double);
  CTOF_CUDA_TRY(cudaFuncSetAttribute(k_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm));
  k_factor<<<nclass, 128, fsm, st>>>(k->d_gram, k->d_lap, nz, 1.0 / (k->scale * k->scale), 0.0, 0, k->d_hinv,
                                     nullptr);
  CTOF_CUDA_TRY(cudaGetLastError());
  CTOF_TRY(contract_admm_prepare(k, st));
  CTOF_CUDA_TRY(cudaStreamSynchronize(st));
  return CTOF_OK;
}

ctof_status build_tikhonov_factors(ctof_kernel_s* k, int slot, double lambda, cudaStream_t st) {
  const int nz = k->nz;
  const size_t fsm = (size_t)2 * nz * (nz + 1) * sizeof(double);
  CTOF_CUDA_TRY(cudaFuncSetAttribute(k_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm));
  k_factor<<<k->nclass, 128, fsm, st>>>(k->d_gram, k->d_lap, nz, 0.0, lambda, 1, k->d_tik_hinv[slot], nullptr);
  CTOF_CUDA_TRY(cudaGetLastError());
  k->tik_lambda[slot] = lambda;
  return CTOF_OK;
}
