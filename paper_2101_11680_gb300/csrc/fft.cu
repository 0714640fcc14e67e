// Lateral 2-D FFTs of the confocal planes (Section 4, "Computational
// Complexity Analysis": the convolution with the K x K blur kernel runs via
// FFTs).  Planes are P x P real (P a power of two, 32..512); spectra are the
// R2C half plane P x (P/2+1) stored frequency-major, f = ky*(P/2+1) + kx, with
// the plane index (time bin or depth) fastest, because the per-frequency
// contraction reads whole T- or Z-vectors of one frequency.
//
// Two passes per direction, through an intermediate inter[row][kx][plane]
// (plane fastest, plane pitch LP = nplanes rounded up to 16):
//   rows    (x axis, real <-> complex): a CTA takes one row index for 16
//           planes; each warp transforms the rows of two planes packed as one
//           complex row and splits them with the Hermitian identities; the 16
//           planes' half spectra leave through shared memory as 128-byte runs
//           of consecutive planes.
//   columns (y axis, complex): a CTA stages 32 columns (32/PB kx x PB
//           consecutive planes) of all rows in shared memory, each warp
//           transforms whole columns; both the intermediate and the
//           frequency-major spectra are read and written in runs of PB planes
//           (PB = 8, 16 or 32, picked per handle by the autotuner).  The
//           transpose between plane-major input planes and frequency-major
//           spectra happens in the row pass's shared-memory tile.
// Each 1-D transform of length P = 32 R lives in one warp: lane l register r
// holds element l + 32 r; an R-point DIF over registers, a twiddle by
// w_P^(l k2), and a 32-point DIF across lanes (shuffles) give element
// R*bitrev5(l) + bitrev_R(r).  Twiddles exp(-2 pi i j/P) are computed on the
// host in double precision and staged in shared memory.
#include <cuda_runtime.h>

#include "ctof_internal.h"

namespace {

// Column-pass tiles hold NC = 32 or 16 columns: KB kx-columns x PB planes;
// the tile shape (NC, PB) is chosen per handle and use by the autotuner
// (tile code PB for NC = 32, 100 + PB for NC = 16: smaller tiles, more CTAs
// per SM).
constexpr int COL_THREADS = 256;
constexpr int ROW_WARPS = 8;

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }
__host__ __device__ constexpr int bitrevc(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r = (r << 1) | ((i >> b) & 1);
  return r;
}

__device__ __forceinline__ int brev5(int l) { return (int)(__brev((unsigned)l) >> 27); }

template <int P, bool INV>
__device__ __forceinline__ float2 tw_get(const float2* tw, int j) {
  float2 w = tw[j & (P - 1)];
  return INV ? make_float2(w.x, -w.y) : w;
}

// Shared twiddle table: the P roots w^j, then per-lane copies of the values
// the lanes need at the same time, so that those reads hit distinct banks:
// [P + s - 1 + l] = w^(l P / 2s) for the cross-lane stage s (l < s), and
// [P + 31 + 32 (k2 - 1) + lane] = w^(lane k2) for the register twiddles.
__host__ __device__ constexpr int tw_count(int P) { return P + 31 + 32 * (P / 32 - 1); }

template <bool INV>
__device__ __forceinline__ float2 tw_conj(float2 w) {
  return INV ? make_float2(w.x, -w.y) : w;
}

// 4- and 8-point DFTs in registers, natural order in and out (w = exp(-2 pi i / n),
// conjugated when INV).
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {  // a * (-i), or a * (+i) when INV
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  const float2 s02 = cadd(x0, x2), d02 = csub(x0, x2), s13 = cadd(x1, x3), d13 = mul_mi<INV>(csub(x1, x3));
  x0 = cadd(s02, s13);
  x2 = csub(s02, s13);
  x1 = cadd(d02, d13);
  x3 = csub(d02, d13);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2 (&x)[8]) {
  float2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6], o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  const float h = 0.70710678118654752f;
  // w8 o1, w8^2 o2, w8^3 o3 with w8 = (1 - i)/sqrt(2) (conjugated when INV)
  const float2 t1 = INV ? make_float2(h * (o1.x - o1.y), h * (o1.x + o1.y))
                        : make_float2(h * (o1.x + o1.y), h * (o1.y - o1.x));
  const float2 t2 = mul_mi<INV>(o2);
  const float2 t3 = INV ? make_float2(-h * (o3.x + o3.y), h * (o3.x - o3.y))
                        : make_float2(h * (o3.y - o3.x), -h * (o3.x + o3.y));
  x[0] = cadd(e0, o0);
  x[4] = csub(e0, o0);
  x[1] = cadd(e1, t1);
  x[5] = csub(e1, t1);
  x[2] = cadd(e2, t2);
  x[6] = csub(e2, t2);
  x[3] = cadd(e3, t3);
  x[7] = csub(e3, t3);
}

// Scratch slots of the 32-point step for P >= 256 (each a permutation of
// [0, P)): S[i][l] (register i, lane l) and S2[i][m1][b]; the rotations keep a
// half-warp's 8-byte accesses on distinct banks (at most 2-way conflicts).
__device__ __forceinline__ int slot_a(int i, int l) { return i * 32 + ((l + 8 * (i & 1)) & 31); }
__device__ __forceinline__ int slot_c(int i, int m1, int b) {
  const int t = 4 * i + m1;
  return t * 8 + (b ^ (t & 7));
}

// Length-P DFT held by one warp (see file comment).  INV selects exp(+...).
// With SCRATCH and P >= 256 (the column passes, whose warps own a tile column
// to use as scratch) the 32-point DFT across the lanes runs as 4 x 8 points in
// registers, with two passes through the scratch (P slots `stride` float2
// apart), instead of five shuffle stages (measured ~10 % faster there; the
// row passes keep the shuffles, which measured faster for them):
//   Z[m1 + 4 m2] = sum_b w8^(b m2) w32^(b m1) sum_a y[b + 8 a] w4^(a m1).
template <int P, bool INV, bool SCRATCH = true>
__device__ __forceinline__ void warp_fft(float2 (&v)[P / 32], int lane, const float2* tw, float2* scr, int stride) {
  constexpr int R = P / 32;
#pragma unroll
  for (int s = R / 2; s >= 1; s >>= 1) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      if ((i & s) == 0) {
        const float2 a = v[i], b = v[i + s];
        v[i] = cadd(a, b);
        v[i + s] = cmul(csub(a, b), tw_get<P, INV>(tw, (i & (s - 1)) * (P / (2 * s))));
      }
    }
  }
#pragma unroll
  for (int i = 1; i < R; ++i) {
    const int k2 = bitrevc(i, ilog2c(R));
    v[i] = cmul(v[i], tw_conj<INV>(tw[P + 31 + 32 * (k2 - 1) + lane]));
  }
  if constexpr (SCRATCH && R >= 8) {
    __syncwarp();  // every lane has read its inputs (callers may pass their input column as scratch)
#pragma unroll
    for (int i = 0; i < R; ++i) scr[slot_a(i, lane) * stride] = v[i];
    __syncwarp();
    const int b = lane & 7;
    float2 t[R / 4][4];
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
      const int i = (lane >> 3) + 4 * q;
#pragma unroll
      for (int a = 0; a < 4; ++a) t[q][a] = scr[slot_a(i, b + 8 * a) * stride];
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
      const int i = (lane >> 3) + 4 * q;
      dft4<INV>(t[q][0], t[q][1], t[q][2], t[q][3]);
#pragma unroll
      for (int m1 = 1; m1 < 4; ++m1) t[q][m1] = cmul(t[q][m1], tw_get<P, INV>(tw, R * b * m1));
#pragma unroll
      for (int m1 = 0; m1 < 4; ++m1) scr[slot_c(i, m1, b) * stride] = t[q][m1];
    }
    __syncwarp();
    const int m1 = lane & 3;
#pragma unroll
    for (int q = 0; q < R / 8; ++q) {
      const int i = (lane >> 2) + 8 * q;
      float2 u[8];
#pragma unroll
      for (int bb = 0; bb < 8; ++bb) u[bb] = scr[slot_c(i, m1, bb) * stride];
      dft8<INV>(u);
#pragma unroll
      for (int m2 = 0; m2 < 8; ++m2) v[8 * q + m2] = u[m2];
    }
    __syncwarp();
  } else {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
      const bool upper = (lane & s) != 0;
      const float2 w = tw_conj<INV>(tw[P + s - 1 + (lane & (s - 1))]);
#pragma unroll
      for (int i = 0; i < R; ++i) {
        float2 o;
        o.x = __shfl_xor_sync(0xffffffffu, v[i].x, s);
        o.y = __shfl_xor_sync(0xffffffffu, v[i].y, s);
        v[i] = upper ? cmul(csub(o, v[i]), w) : cadd(v[i], o);
      }
    }
  }
}

// Output position of register i of lane `lane` after warp_fft<P, INV, SCRATCH>.
template <int P, bool SCRATCH = true>
__device__ __forceinline__ int out_pos(int lane, int i) {
  constexpr int R = P / 32;
  if constexpr (SCRATCH && R >= 8) {
    // register 8 q + m2 of lane L: k1 = bitrev_R((L >> 2) + 8 q), k2 = (L & 3) + 4 m2
    return bitrevc((lane >> 2) + 8 * (i >> 3), ilog2c(R)) + R * ((lane & 3) + 4 * (i & 7));
  } else {
    return R * brev5(lane) + bitrevc(i, ilog2c(R));
  }
}

// Shared-memory slot of transform element e.  A warp writes its R registers
// to elements R*bitrev5(lane) + i', i.e. 32 elements R apart, which would all
// fall in two banks; XOR-ing the low log2(R) bits with the next ones spreads
// them over all banks.  A permutation within each aligned block of R elements.
template <int P>
__device__ __forceinline__ int sw_pos(int e) {
  constexpr int R = P / 32;
  return e ^ ((e / R) & (R - 1));
}

template <int P>
__device__ __forceinline__ void stage_twiddles(float2* s_tw, const float2* tw) {
  for (int i = threadIdx.x; i < tw_count(P); i += blockDim.x) {
    int j;
    if (i < P) {
      j = i;
    } else if (i < P + 31) {
      const int e = i - P;
      int s = 1;
      while (2 * s - 1 <= e) s *= 2;  // stage s holds entries s-1 .. 2s-2
      j = (e - (s - 1)) * (P / (2 * s));
    } else {
      const int e = i - P - 31;
      j = ((e & 31) * (e / 32 + 1)) & (P - 1);
    }
    s_tw[i] = tw[j];
  }
}

// ---------------------------------------------------------------- rows ----

constexpr int RP = 2 * ROW_WARPS;  // planes per row-pass CTA

__host__ __device__ inline int plane_ld(int nplanes) { return (nplanes + RP - 1) / RP * RP; }

// Half spectra of the CTA's planes for one row: s_h[kx][plane] (pitch RP + 1).
constexpr int SH_LD = RP + 1;

template <int P>
__device__ __forceinline__ void split_to_tile(const float2* buf, int lane, float2* s_h, int c0) {
  for (int kk = lane; kk <= P / 2; kk += 32) {
    const float2 zk = buf[sw_pos<P>(kk)];
    const float2 zm = buf[sw_pos<P>((P - kk) & (P - 1))];
    s_h[kk * SH_LD + c0] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    s_h[kk * SH_LD + c0 + 1] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
  }
}

// Z[n] = A[n] + i B[n] from the half spectra in tile columns c0, c0 + 1.
template <int P>
__device__ __forceinline__ void load_pair_from_tile(float2 (&v)[P / 32], const float2* s_h, int c0, int lane) {
  constexpr int R = P / 32;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int n = lane + 32 * i;
    float2 A, B;
    if (n <= P / 2) {
      A = s_h[n * SH_LD + c0];
      B = s_h[n * SH_LD + c0 + 1];
    } else {
      A = cconj(s_h[(P - n) * SH_LD + c0]);
      B = cconj(s_h[(P - n) * SH_LD + c0 + 1]);
    }
    v[i] = make_float2(A.x - B.y, A.y + B.x);
  }
}

template <int P>
__device__ __forceinline__ void store_tile(const float2* s_h, float2* __restrict__ inter, int r, int hp, int LP,
                                           int pl0, int nplanes) {
  for (int idx = threadIdx.x; idx < (P / 2 + 1) * RP; idx += blockDim.x) {
    const int kk = idx / RP, pl = idx - kk * RP;
    if (pl0 + pl < nplanes) inter[((size_t)r * hp + kk) * LP + pl0 + pl] = s_h[kk * SH_LD + pl];
  }
}

template <int P>
__device__ __forceinline__ void load_tile(float2* s_h, const float2* __restrict__ inter, int r, int hp, int LP,
                                          int pl0, int nplanes) {
  for (int idx = threadIdx.x; idx < (P / 2 + 1) * RP; idx += blockDim.x) {
    const int kk = idx / RP, pl = idx - kk * RP;
    s_h[kk * SH_LD + pl] =
        pl0 + pl < nplanes ? inter[((size_t)r * hp + kk) * LP + pl0 + pl] : make_float2(0.f, 0.f);
  }
}

// Forward R2C of rows: in[plane][row][ld_in] (first cols_in columns, zero beyond)
// -> inter[row][kx][LP].
template <int P>
__global__ void __launch_bounds__(ROW_WARPS * 32) k_rows_fwd(const float* __restrict__ in, int nplanes, int rows,
                                                             int cols_in, int ld_in, float2* __restrict__ inter,
                                                             int hp, const float2* __restrict__ tw) {
  constexpr int R = P / 32;
  extern __shared__ float2 smem[];
  float2* s_tw = smem;
  float2* s_h = smem + tw_count(P);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* buf = s_h + (P / 2 + 1) * SH_LD + warp * (P + 2);
  stage_twiddles<P>(s_tw, tw);
  __syncthreads();
  const int LP = plane_ld(nplanes), nblk = LP / RP;
  for (int job = blockIdx.x; job < rows * nblk; job += gridDim.x) {
    const int r = job / nblk, pl0 = (job - r * nblk) * RP;
    const int p0 = pl0 + 2 * warp, p1 = p0 + 1;
    const float* r0 = in + ((size_t)p0 * rows + r) * ld_in;
    const float* r1 = in + ((size_t)p1 * rows + r) * ld_in;
    float2 v[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int n = lane + 32 * i;
      const float a = (p0 < nplanes && n < cols_in) ? r0[n] : 0.f;
      const float b = (p1 < nplanes && n < cols_in) ? r1[n] : 0.f;
      v[i] = make_float2(a, b);
    }
    warp_fft<P, false, false>(v, lane, s_tw, buf, 1);
#pragma unroll
    for (int i = 0; i < R; ++i) buf[sw_pos<P>(out_pos<P, false>(lane, i))] = v[i];
    __syncwarp();
    split_to_tile<P>(buf, lane, s_h, 2 * warp);
    __syncthreads();
    store_tile<P>(s_h, inter, r, hp, LP, pl0, nplanes);
    __syncthreads();
  }
}

// Inverse C2R of rows: inter[row][kx][LP] -> out[plane][row][ld_out] (first cols_out columns), x scale.
template <int P>
__global__ void __launch_bounds__(ROW_WARPS * 32) k_rows_inv(const float2* __restrict__ inter, int nplanes,
                                                             int rows, int hp, int cols_out, float* __restrict__ out,
                                                             int ld_out, float scale,
                                                             const float2* __restrict__ tw) {
  constexpr int R = P / 32;
  extern __shared__ float2 smem[];
  float2* s_tw = smem;
  float2* s_h = smem + tw_count(P);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* buf = s_h + (P / 2 + 1) * SH_LD + warp * (P + 2);
  stage_twiddles<P>(s_tw, tw);
  const int LP = plane_ld(nplanes), nblk = LP / RP;
  for (int job = blockIdx.x; job < rows * nblk; job += gridDim.x) {
    const int r = job / nblk, pl0 = (job - r * nblk) * RP;
    const int p0 = pl0 + 2 * warp, p1 = p0 + 1;
    load_tile<P>(s_h, inter, r, hp, LP, pl0, nplanes);
    __syncthreads();
    float2 v[R];
    load_pair_from_tile<P>(v, s_h, 2 * warp, lane);
    warp_fft<P, true, false>(v, lane, s_tw, buf, 1);
#pragma unroll
    for (int i = 0; i < R; ++i) buf[sw_pos<P>(out_pos<P, false>(lane, i))] = v[i];
    __syncwarp();
    for (int c = lane; c < cols_out; c += 32) {
      const float2 z = buf[sw_pos<P>(c)];
      if (p0 < nplanes) out[((size_t)p0 * rows + r) * ld_out + c] = z.x * scale;
      if (p1 < nplanes) out[((size_t)p1 * rows + r) * ld_out + c] = z.y * scale;
    }
    __syncthreads();
  }
}

// ADMM T side, per measurement row y and pair of time bins t:
//   Kx   = C2R(row spectra) on the N scan columns
//   a1   = Kx + u1;  v1 = (m/scale + rho a1) / (1 + rho);  u1 <- a1 - v1
//   c    = (v1 - u1) - Kx = 2 v1 - a1 - Kx      (zero off the scan)
//   row spectra <- R2C(c zero-padded to P)
// so that FFT(v1 - u1) = K x_hat + c_hat without a transform of the full
// P x P plane.  m, u1: [nt][n][n]; inter: [n][kx][LP] in place.
template <int P>
__global__ void __launch_bounds__(ROW_WARPS * 32) k_rows_admm_t(float2* __restrict__ inter, int nplanes, int n,
                                                                int hp, const float* __restrict__ m,
                                                                float* __restrict__ u1, float scale, float inv_s,
                                                                float rho, const float2* __restrict__ tw) {
  constexpr int R = P / 32;
  extern __shared__ float2 smem[];
  float2* s_tw = smem;
  float2* s_h = smem + tw_count(P);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* buf = s_h + (P / 2 + 1) * SH_LD + warp * (P + 2);
  stage_twiddles<P>(s_tw, tw);
  const float inv1r = 1.0f / (1.0f + rho);
  const int LP = plane_ld(nplanes), nblk = LP / RP;
  for (int job = blockIdx.x; job < n * nblk; job += gridDim.x) {
    const int r = job / nblk, pl0 = (job - r * nblk) * RP;
    const int p0 = pl0 + 2 * warp, p1 = p0 + 1;
    const bool has0 = p0 < nplanes, has1 = p1 < nplanes;
    load_tile<P>(s_h, inter, r, hp, LP, pl0, nplanes);
    __syncthreads();
    float2 v[R];
    load_pair_from_tile<P>(v, s_h, 2 * warp, lane);
    warp_fft<P, true, false>(v, lane, s_tw, buf, 1);
#pragma unroll
    for (int i = 0; i < R; ++i) buf[sw_pos<P>(out_pos<P, false>(lane, i))] = v[i];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int c = lane + 32 * i;
      float2 cc = make_float2(0.f, 0.f);
      if (c < n) {
        const float2 kx = cscale(buf[sw_pos<P>(c)], scale);
        if (has0) {
          const size_t idx = ((size_t)p0 * n + r) * n + c;
          const float a1 = kx.x + u1[idx];
          const float v1 = (m[idx] * inv_s + rho * a1) * inv1r;
          u1[idx] = a1 - v1;
          cc.x = 2.f * v1 - a1 - kx.x;
        }
        if (has1) {
          const size_t idx = ((size_t)p1 * n + r) * n + c;
          const float a1 = kx.y + u1[idx];
          const float v1 = (m[idx] * inv_s + rho * a1) * inv1r;
          u1[idx] = a1 - v1;
          cc.y = 2.f * v1 - a1 - kx.y;
        }
      }
      v[i] = cc;
    }
    __syncwarp();
    warp_fft<P, false, false>(v, lane, s_tw, buf, 1);
#pragma unroll
    for (int i = 0; i < R; ++i) buf[sw_pos<P>(out_pos<P, false>(lane, i))] = v[i];
    __syncwarp();
    __syncthreads();  // every warp is done reading s_h
    split_to_tile<P>(buf, lane, s_h, 2 * warp);
    __syncthreads();
    store_tile<P>(s_h, inter, r, hp, LP, pl0, nplanes);
    __syncthreads();
  }
}

// ------------------------------------------------------------- columns ----

// Forward C2C along y: inter[row][kx][LP] (rows_in rows, zero beyond) -> out[ky h + kx][ldf].
template <int P, int PB, int NC>
__global__ void __launch_bounds__(COL_THREADS) k_cols_fwd(const float2* __restrict__ inter, int nplanes,
                                                          int rows_in, int h, int hp,
                                                          float2* __restrict__ out, int ldf,
                                                          const float2* __restrict__ tw) {
  constexpr int R = P / 32;
  constexpr int KB = NC / PB;
  constexpr int LDT = NC + 1;
  extern __shared__ float2 smem[];
  float2* s_tw = smem;
  float2* tile = smem + tw_count(P);
  const int kx0 = blockIdx.x * KB, pl0 = blockIdx.y * PB;
  const int LP = plane_ld(nplanes);
  stage_twiddles<P>(s_tw, tw);
  for (int idx = threadIdx.x; idx < rows_in * NC; idx += COL_THREADS) {
    const int row = idx / NC, cc = idx % NC;
    const int kx = kx0 + cc / PB, pl = pl0 + cc % PB;
    float2 val = make_float2(0.f, 0.f);
    if (kx < h && pl < nplanes) val = inter[((size_t)row * hp + kx) * LP + pl];
    tile[row * LDT + cc] = val;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = warp; c < NC; c += COL_THREADS / 32) {
    float2 v[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int y = lane + 32 * i;
      v[i] = y < rows_in ? tile[y * LDT + c] : make_float2(0.f, 0.f);
    }
    warp_fft<P, false>(v, lane, s_tw, tile + c, LDT);
#pragma unroll
    for (int i = 0; i < R; ++i) tile[sw_pos<P>(out_pos<P>(lane, i)) * LDT + c] = v[i];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < P * NC; idx += COL_THREADS) {
    const int ky = idx / NC, cc = idx % NC;
    const int kx = kx0 + cc / PB, pl = pl0 + cc % PB;
    if (kx < h && pl < nplanes) out[((size_t)ky * h + kx) * ldf + pl] = tile[sw_pos<P>(ky) * LDT + cc];
  }
}

// Inverse C2C along y: in[ky h + kx][ldf] -> inter[row][kx][LP] for the first rows_out rows.
template <int P, int PB, int NC>
__global__ void __launch_bounds__(COL_THREADS) k_cols_inv(const float2* __restrict__ in, int ldf, int nplanes,
                                                          int rows_out, int h, int hp,
                                                          float2* __restrict__ inter,
                                                          const float2* __restrict__ tw) {
  constexpr int R = P / 32;
  constexpr int KB = NC / PB;
  constexpr int LDT = NC + 1;
  extern __shared__ float2 smem[];
  float2* s_tw = smem;
  float2* tile = smem + tw_count(P);
  const int kx0 = blockIdx.x * KB, pl0 = blockIdx.y * PB;
  const int LP = plane_ld(nplanes);
  stage_twiddles<P>(s_tw, tw);
  for (int idx = threadIdx.x; idx < P * NC; idx += COL_THREADS) {
    const int ky = idx / NC, cc = idx % NC;
    const int kx = kx0 + cc / PB, pl = pl0 + cc % PB;
    float2 val = make_float2(0.f, 0.f);
    if (kx < h && pl < nplanes) val = in[((size_t)ky * h + kx) * ldf + pl];
    tile[ky * LDT + cc] = val;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = warp; c < NC; c += COL_THREADS / 32) {
    float2 v[R];
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = tile[(lane + 32 * i) * LDT + c];
    __syncwarp();
    warp_fft<P, true>(v, lane, s_tw, tile + c, LDT);
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int y = out_pos<P>(lane, i);
      if (y < rows_out) tile[sw_pos<P>(y) * LDT + c] = v[i];
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < rows_out * NC; idx += COL_THREADS) {
    const int row = idx / NC, cc = idx % NC;
    const int kx = kx0 + cc / PB, pl = pl0 + cc % PB;
    if (kx < h && pl < nplanes) inter[((size_t)row * hp + kx) * LP + pl] = tile[sw_pos<P>(row) * LDT + cc];
  }
}

// ------------------------------------------------------------ launchers ----

size_t row_smem(int p) {
  return (size_t)(tw_count(p) + (p / 2 + 1) * SH_LD + ROW_WARPS * (p + 2)) * sizeof(float2);
}
size_t col_smem(int p, int nc) { return (size_t)(tw_count(p) + p * (nc + 1)) * sizeof(float2); }

template <typename F>
cudaError_t allow_smem(F* fn, size_t bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

int row_grid(int rows, int nplanes) {
  const int jobs = rows * (plane_ld(nplanes) / RP);
  const int cap = 152 * 8;
  return jobs < 1 ? 1 : (jobs > cap ? cap : jobs);
}

#define CTOF_P_SWITCH(p, ...)                                    \
  switch (p) {                                                   \
    case 32: { constexpr int P_ = 32; __VA_ARGS__; } break;      \
    case 64: { constexpr int P_ = 64; __VA_ARGS__; } break;      \
    case 128: { constexpr int P_ = 128; __VA_ARGS__; } break;    \
    case 256: { constexpr int P_ = 256; __VA_ARGS__; } break;    \
    case 512: { constexpr int P_ = 512; __VA_ARGS__; } break;    \
    default: return CTOF_EUNSUPPORTED;                           \
  }
}  // namespace

ctof_status fft_rows_forward(const ctof_kernel_s* k, const float* in, int nplanes, int rows, int cols_in,
                             int ld_in, float2* inter, cudaStream_t st) {
  if (nplanes <= 0 || rows <= 0) return CTOF_OK;
  const size_t sm = row_smem(k->p);
  CTOF_P_SWITCH(k->p, {
    CTOF_CUDA_TRY(allow_smem(k_rows_fwd<P_>, sm));
    k_rows_fwd<P_><<<row_grid(rows, nplanes), ROW_WARPS * 32, sm, st>>>(in, nplanes, rows, cols_in, ld_in, inter,
                                                                         k->hp, k->d_tw);
  });
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status fft_rows_inverse(const ctof_kernel_s* k, const float2* inter, int nplanes, int rows, int cols_out,
                             float* out, int ld_out, cudaStream_t st) {
  if (nplanes <= 0 || rows <= 0) return CTOF_OK;
  const size_t sm = row_smem(k->p);
  const float scale = 1.0f / ((float)k->p * (float)k->p);
  CTOF_P_SWITCH(k->p, {
    CTOF_CUDA_TRY(allow_smem(k_rows_inv<P_>, sm));
    k_rows_inv<P_><<<row_grid(rows, nplanes), ROW_WARPS * 32, sm, st>>>(inter, nplanes, rows, k->hp, cols_out, out,
                                                                         ld_out, scale, k->d_tw);
  });
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status fft_rows_admm_t(const ctof_kernel_s* k, float2* inter, const float* m, float* u1, float inv_scale,
                            float rho, cudaStream_t st) {
  const size_t sm = row_smem(k->p);
  const float scale = 1.0f / ((float)k->p * (float)k->p);
  CTOF_P_SWITCH(k->p, {
    CTOF_CUDA_TRY(allow_smem(k_rows_admm_t<P_>, sm));
    k_rows_admm_t<P_><<<row_grid(k->n, k->nt), ROW_WARPS * 32, sm, st>>>(inter, k->nt, k->n, k->hp, m, u1, scale,
                                                                          inv_scale, rho, k->d_tw);
  });
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

#define CTOF_COLS_LAUNCH(KERN, ...)                                                          \
  do {                                                                                       \
    const int pb = code >= 100 ? code - 100 : code, nc = code >= 100 ? 16 : 32;              \
    const size_t sm = col_smem(k->p, nc);                                                    \
    dim3 grid(ctof_div_up(k->h, nc / pb), ctof_div_up(nplanes, pb));                        \
    switch (code) {                                                                          \
      case 32:                                                                               \
        CTOF_P_SWITCH(k->p, {                                                                \
          CTOF_CUDA_TRY(allow_smem(KERN<P_, 32, 32>, sm));                                   \
          KERN<P_, 32, 32><<<grid, COL_THREADS, sm, st>>>(__VA_ARGS__);                      \
        });                                                                                  \
        break;                                                                               \
      case 16:                                                                               \
        CTOF_P_SWITCH(k->p, {                                                                \
          CTOF_CUDA_TRY(allow_smem(KERN<P_, 16, 32>, sm));                                   \
          KERN<P_, 16, 32><<<grid, COL_THREADS, sm, st>>>(__VA_ARGS__);                      \
        });                                                                                  \
        break;                                                                               \
      case 116:                                                                              \
        CTOF_P_SWITCH(k->p, {                                                                \
          CTOF_CUDA_TRY(allow_smem(KERN<P_, 16, 16>, sm));                                   \
          KERN<P_, 16, 16><<<grid, COL_THREADS, sm, st>>>(__VA_ARGS__);                      \
        });                                                                                  \
        break;                                                                               \
      case 108:                                                                              \
        CTOF_P_SWITCH(k->p, {                                                                \
          CTOF_CUDA_TRY(allow_smem(KERN<P_, 8, 16>, sm));                                    \
          KERN<P_, 8, 16><<<grid, COL_THREADS, sm, st>>>(__VA_ARGS__);                       \
        });                                                                                  \
        break;                                                                               \
      default:                                                                               \
        CTOF_P_SWITCH(k->p, {                                                                \
          CTOF_CUDA_TRY(allow_smem(KERN<P_, 8, 32>, sm));                                    \
          KERN<P_, 8, 32><<<grid, COL_THREADS, sm, st>>>(__VA_ARGS__);                       \
        });                                                                                  \
    }                                                                                        \
  } while (0)

ctof_status fft_cols_forward_pb(const ctof_kernel_s* k, const float2* inter, int nplanes, int rows_in, float2* out,
                                int ldf, int code, cudaStream_t st) {
  if (nplanes <= 0) return CTOF_OK;
  CTOF_COLS_LAUNCH(k_cols_fwd, inter, nplanes, rows_in, k->h, k->hp, out, ldf, k->d_tw);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status fft_cols_forward(const ctof_kernel_s* k, const float2* inter, int nplanes, int rows_in, float2* out,
                             int ldf, cudaStream_t st) {
  const int pb = (nplanes == k->nt) ? k->tune_pb[0] : k->tune_pb[2];
  return fft_cols_forward_pb(k, inter, nplanes, rows_in, out, ldf, pb, st);
}

ctof_status fft_cols_inverse_pb(const ctof_kernel_s* k, const float2* in, int ldf, int nplanes, int rows_out,
                                float2* inter, int code, cudaStream_t st) {
  if (nplanes <= 0) return CTOF_OK;
  CTOF_COLS_LAUNCH(k_cols_inv, in, ldf, nplanes, rows_out, k->h, k->hp, inter, k->d_tw);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status fft_cols_inverse(const ctof_kernel_s* k, const float2* in, int ldf, int nplanes, int rows_out,
                             float2* inter, cudaStream_t st) {
  const int pb = (nplanes == k->nt) ? k->tune_pb[1] : k->tune_pb[3];
  return fft_cols_inverse_pb(k, in, ldf, nplanes, rows_out, inter, pb, st);
}

size_t fft_inter_elems(const ctof_kernel_s* k, int nplanes, int rows) {
  return (size_t)rows * k->hp * plane_ld(nplanes);
}

ctof_status fft_forward_planes(const ctof_kernel_s* k, const float* in, int nplanes, int rows_in, int cols_in,
                               int ld_in, float2* inter, float2* out, int ldf, cudaStream_t st) {
  CTOF_TRY(fft_rows_forward(k, in, nplanes, rows_in, cols_in, ld_in, inter, st));
  return fft_cols_forward(k, inter, nplanes, rows_in, out, ldf, st);
}

ctof_status fft_inverse_planes(const ctof_kernel_s* k, const float2* in, int ldf, int nplanes, int rows_out,
                               int cols_out, float2* inter, float* out, int ld_out, cudaStream_t st) {
  CTOF_TRY(fft_cols_inverse(k, in, ldf, nplanes, rows_out, inter, st));
  return fft_rows_inverse(k, inter, nplanes, rows_out, cols_out, out, ld_out, st);
}
