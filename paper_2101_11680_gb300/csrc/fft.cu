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

#include <math.h>

#include "bulk.cuh"
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

// Twiddle table, built on the host in this layout and copied to shared memory
// as is: the P roots w^j, then per-lane copies of the values the lanes need at
// the same time, so that those reads hit distinct banks:
// [P + s - 1 + l] = w^(l P / 2s) for the cross-lane stage s (l < s), and
// [P + 31 + 32 (k - 1) + lane] = w^(lane k) for the register twiddles;
// padded to an even count (a multiple of 16 bytes).
__host__ __device__ constexpr int tw_count(int P) { return P + 31 + 32 * (P / 32 - 1); }
__host__ __device__ constexpr int tw_pad(int P) { return (tw_count(P) + 1) & ~1; }

template <bool INV>
__device__ __forceinline__ float2 tw_conj(float2 w) {
  return INV ? make_float2(w.x, -w.y) : w;
}

// Transform values: one column (float2) or two adjacent columns handled by
// the same lane (cpair, one 16-byte shared-memory access).
struct cpair {
  float2 a, b;
};
__device__ __forceinline__ float2 vadd(float2 x, float2 y) { return cadd(x, y); }
__device__ __forceinline__ cpair vadd(cpair x, cpair y) { return {cadd(x.a, y.a), cadd(x.b, y.b)}; }
__device__ __forceinline__ float2 vsub(float2 x, float2 y) { return csub(x, y); }
__device__ __forceinline__ cpair vsub(cpair x, cpair y) { return {csub(x.a, y.a), csub(x.b, y.b)}; }
__device__ __forceinline__ float2 vmul(float2 x, float2 w) { return cmul(x, w); }
__device__ __forceinline__ cpair vmul(cpair x, float2 w) { return {cmul(x.a, w), cmul(x.b, w)}; }
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {  // a * (-i), or a * (+i) when INV
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
template <bool INV>
__device__ __forceinline__ float2 vmi(float2 a) {
  return mul_mi<INV>(a);
}
template <bool INV>
__device__ __forceinline__ cpair vmi(cpair a) {
  return {mul_mi<INV>(a.a), mul_mi<INV>(a.b)};
}
__device__ __forceinline__ void vld(float2& v, const float2* p) { v = *p; }
__device__ __forceinline__ void vld(cpair& v, const float2* p) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v.a = make_float2(q.x, q.y);
  v.b = make_float2(q.z, q.w);
}
__device__ __forceinline__ void vst(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void vst(float2* p, cpair v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.a.x, v.a.y, v.b.x, v.b.y);
}
__device__ __forceinline__ void vzero(float2& v) { v = make_float2(0.f, 0.f); }
__device__ __forceinline__ void vzero(cpair& v) { v.a = v.b = make_float2(0.f, 0.f); }
__device__ __forceinline__ float2 shfl2(float2 v, int s) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, s), __shfl_xor_sync(0xffffffffu, v.y, s));
}
__device__ __forceinline__ float2 vshfl(float2 v, int s) { return shfl2(v, s); }
__device__ __forceinline__ cpair vshfl(cpair v, int s) { return {shfl2(v.a, s), shfl2(v.b, s)}; }

// exp(-2 pi i j / n) given as (re, im); conjugated when INV.
template <bool INV>
__device__ __forceinline__ float2 root(float re, float im) {
  return make_float2(re, INV ? -im : im);
}

// 2-, 4-, 8- and 16-point DFTs in registers with constant twiddles, natural
// order in and out (w = exp(-2 pi i / n), conjugated when INV).
template <bool INV, typename T>
__device__ __forceinline__ void dft2(T& x0, T& x1) {
  const T s = vadd(x0, x1);
  x1 = vsub(x0, x1);
  x0 = s;
}

template <bool INV, typename T>
__device__ __forceinline__ void dft4(T& x0, T& x1, T& x2, T& x3) {
  const T s02 = vadd(x0, x2), d02 = vsub(x0, x2), s13 = vadd(x1, x3), d13 = vmi<INV>(vsub(x1, x3));
  x0 = vadd(s02, s13);
  x2 = vsub(s02, s13);
  x1 = vadd(d02, d13);
  x3 = vsub(d02, d13);
}

// Radix-2 step over the 4-point DFTs E, O of the even and odd samples:
// X[k] = E[k] + w8^k O[k], X[k + 4] = E[k] - w8^k O[k].
template <bool INV, typename T>
__device__ __forceinline__ void dft8(T (&x)[8]) {
  T e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6], o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  constexpr float h = 0.70710678118654752f;
  o1 = vmul(o1, root<INV>(h, -h));
  o2 = vmi<INV>(o2);
  o3 = vmul(o3, root<INV>(-h, -h));
  x[0] = vadd(e0, o0);
  x[4] = vsub(e0, o0);
  x[1] = vadd(e1, o1);
  x[5] = vsub(e1, o1);
  x[2] = vadd(e2, o2);
  x[6] = vsub(e2, o2);
  x[3] = vadd(e3, o3);
  x[7] = vsub(e3, o3);
}

// 4 x 4: X[k1 + 4 k2] = sum_n2 w4^(n2 k2) w16^(n2 k1) sum_n1 x[4 n1 + n2] w4^(n1 k1).
template <bool INV, typename T>
__device__ __forceinline__ void dft16(T (&x)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
  // x[n2 + 4 k1] now holds the inner sum for (n2, k1)
  constexpr float c1 = 0.92387953251128676f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
  x[5] = vmul(x[5], root<INV>(c1, -s1));    // w16^1
  x[9] = vmul(x[9], root<INV>(h, -h));      // w16^2
  x[13] = vmul(x[13], root<INV>(s1, -c1));  // w16^3
  x[6] = vmul(x[6], root<INV>(h, -h));      // w16^2
  x[10] = vmi<INV>(x[10]);                  // w16^4
  x[14] = vmul(x[14], root<INV>(-h, -h));   // w16^6
  x[7] = vmul(x[7], root<INV>(s1, -c1));    // w16^3
  x[11] = vmul(x[11], root<INV>(-h, -h));   // w16^6
  x[15] = vmul(x[15], root<INV>(-c1, s1));  // w16^9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
  T y[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) y[k1 + 4 * k2] = x[4 * k1 + k2];
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = y[i];
}

template <int R, bool INV, typename T>
__device__ __forceinline__ void reg_dft(T (&v)[R]) {
  if constexpr (R == 2) {
    dft2<INV>(v[0], v[1]);
  } else if constexpr (R == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    dft8<INV>(v);
  } else if constexpr (R == 16) {
    dft16<INV>(v);
  }
}

// Scratch slots of the 32-point step for P >= 256 (each a permutation of
// [0, P)): S[i][l] (register i, lane l) and S2[i][m1][b].  Eight consecutive
// lanes always touch eight slots that are distinct mod 8 (conflict-free
// 16-byte accesses on the column tile's pitch); the rotation in S keeps a
// half-warp's 8-byte accesses on distinct banks for odd pitches.
__device__ __forceinline__ int slot_a(int i, int l) { return i * 32 + ((l + 8 * (i & 1)) & 31); }
__device__ __forceinline__ int slot_c(int i, int m1, int b) {
  const int t = 4 * i + m1;
  return t * 8 + (b ^ (t & 7));
}

// Length-P DFT held by one warp, P = 32 R: lane l register i holds element
// l + 32 i (of one column, or of each of two columns).  X[k1 + R k2] =
// sum_l w32^(l k2) w_P^(l k1) sum_i x[l + 32 i] w_R^(i k1): an R-point DFT
// over the registers (register i then holds k1 = i), the twiddle w_P^(l k1),
// and a 32-point DFT across the lanes.  INV selects exp(+...).
// With SCRATCH and P >= 256 (the column passes, whose warps own a tile column
// pair to use as scratch) the 32-point DFT across the lanes runs as 4 x 8
// points in registers with two passes through the scratch (P slots `stride`
// float2 apart):
//   Z[m1 + 4 m2] = sum_b w8^(b m2) w32^(b m1) sum_a y[b + 8 a] w4^(a m1);
// otherwise as five shuffle stages (DIF, outputs in bit-reversed lane order).
template <int P, bool INV, bool SCRATCH = true, typename T>
__device__ __forceinline__ void warp_fft(T (&v)[P / 32], int lane, const float2* tw, float2* scr, int stride) {
  constexpr int R = P / 32;
  reg_dft<R, INV>(v);
#pragma unroll
  for (int i = 1; i < R; ++i) v[i] = vmul(v[i], tw_conj<INV>(tw[P + 31 + 32 * (i - 1) + lane]));
  if constexpr (SCRATCH && R >= 8) {
    __syncwarp();  // every lane has read its inputs (callers may pass their input column as scratch)
#pragma unroll
    for (int i = 0; i < R; ++i) vst(scr + slot_a(i, lane) * stride, v[i]);
    __syncwarp();
    const int b = lane & 7;
    T t[R / 4][4];
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
      const int i = (lane >> 3) + 4 * q;
#pragma unroll
      for (int a = 0; a < 4; ++a) vld(t[q][a], scr + slot_a(i, b + 8 * a) * stride);
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
      const int i = (lane >> 3) + 4 * q;
      dft4<INV>(t[q][0], t[q][1], t[q][2], t[q][3]);
#pragma unroll
      for (int m1 = 1; m1 < 4; ++m1) t[q][m1] = vmul(t[q][m1], tw_get<P, INV>(tw, R * b * m1));
#pragma unroll
      for (int m1 = 0; m1 < 4; ++m1) vst(scr + slot_c(i, m1, b) * stride, t[q][m1]);
    }
    __syncwarp();
    const int m1 = lane & 3;
#pragma unroll
    for (int q = 0; q < R / 8; ++q) {
      const int i = (lane >> 2) + 8 * q;
      T u[8];
#pragma unroll
      for (int bb = 0; bb < 8; ++bb) vld(u[bb], scr + slot_c(i, m1, bb) * stride);
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
        const T o = vshfl(v[i], s);
        v[i] = upper ? vmul(vsub(o, v[i]), w) : vadd(v[i], o);
      }
    }
  }
}

// Output position of register i of lane `lane` after warp_fft<P, INV, SCRATCH>.
template <int P, bool SCRATCH = true>
__device__ __forceinline__ int out_pos(int lane, int i) {
  constexpr int R = P / 32;
  if constexpr (SCRATCH && R >= 8) {
    // register 8 q + m2 of lane L: k1 = (L >> 2) + 8 q, k2 = (L & 3) + 4 m2
    return (lane >> 2) + 8 * (i >> 3) + R * ((lane & 3) + 4 * (i & 7));
  } else {
    return i + R * brev5(lane);
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
  for (int i = threadIdx.x; i < tw_pad(P); i += blockDim.x) s_tw[i] = tw[i];
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
  float2* s_h = smem + tw_pad(P);
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
  float2* s_h = smem + tw_pad(P);
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
  float2* s_h = smem + tw_pad(P);
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

// Column-pass tile: P rows x NC columns (KB = NC / PB kx-columns x PB
// consecutive planes), row pitch NC + 2 float2: rows start on 16-byte
// boundaries (targets and sources of bulk copies), and eight rows that are
// distinct mod 8 put a quarter-warp's 16-byte accesses on distinct bank
// groups.  Each warp transforms two adjacent columns at once (cpair).
template <int NC>
__host__ __device__ constexpr int col_ld() {
  return NC + 2;
}

// Tile row of transform output e: a permutation of [0, P) under which the
// eight outputs that eight consecutive lanes write with one register land in
// rows distinct mod 8.  4 x 8 path (R >= 8): e = k1 + R k2 with k1 = (L >> 2)
// + 8 q and k2 = (L & 3) + 4 m2, so bits 1-2 of k1 (zero there) take k2's low
// bits.  Shuffle path: e = i + 4 R rev3(L), so the low bits take the three
// bits above 4 R.
template <int P>
__device__ __forceinline__ int col_row(int e) {
  constexpr int R = P / 32;
  if constexpr (R >= 8) {
    return e ^ (((e / R) & 3) << 1);
  } else if constexpr (R >= 2) {
    return e ^ ((e >> (ilog2c(R) + 2)) & 7);
  } else {
    return e ^ ((e >> 3) & 3);
  }
}

// Shared memory of a column pass: [mbarrier, 16 B][twiddles][tile].
__host__ __device__ constexpr size_t col_smem_bytes(int P, int NC) {
  return 16 + ((size_t)tw_pad(P) + (size_t)P * (NC + 2)) * sizeof(float2);
}

// Stages the tile's runs (`nrun` runs of `run` bytes; run r goes from
// src(r) to dst(r)) and the twiddles by bulk copies completing on one
// mbarrier.  Block-wide; false (and the handle's status flag set) when the
// copies did not land within max_polls polls.
template <int P, typename Src, typename Dst>
__device__ __forceinline__ bool col_stage_in(uint64_t* bar, float2* s_tw, const float2* tw, int nrun, unsigned run,
                                             Src src, Dst dst, int* flag, long long max_polls) {
  if (threadIdx.x == 0) {
    bulk::bar_init(bar, 1);
    bulk::arrive_expect(bar, (unsigned)nrun * run + tw_pad(P) * (unsigned)sizeof(float2));
    bulk::g2s(s_tw, tw, tw_pad(P) * sizeof(float2), bar);
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nrun; r += COL_THREADS) bulk::g2s(dst(r), src(r), run, bar);
  const bool ok = __syncthreads_and(bulk::wait(bar, 0, max_polls));
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(flag, 1);
    bulk::wait(bar, 0, bulk::DRAIN_POLLS);
  }
  return ok;
}

// Writes the tile's runs back: `nrun` runs of np planes, run r from src(r) to
// dst(r); the even part by bulk copies, an odd last plane by a plain store.
template <typename Src, typename Dst>
__device__ __forceinline__ void col_stage_out(int nrun, int np, Src src, Dst dst) {
  bulk::fence_smem();  // the tile writes of this thread, before the copies read them
  __syncthreads();
  const int ne = np & ~1;
  bool issued = false;
  for (int r = threadIdx.x; r < nrun; r += COL_THREADS) {
    const float2* s = src(r);
    float2* d = dst(r);
    if (ne) {
      bulk::s2g(d, s, (unsigned)ne * sizeof(float2));
      issued = true;
    }
    if (np & 1) d[ne] = s[ne];
  }
  if (issued) {
    bulk::commit();
    bulk::wait_read_all();
  }
}

// Forward C2C along y: inter[row][kx][LP] (rows_in rows, zero beyond) -> out[ky h + kx][ldf].
// BULK: tile staged in and out by bulk copies (16-byte aligned buffers, even
// ldf); otherwise element by element.
template <int P, int PB, int NC, bool BULK>
__global__ void __launch_bounds__(COL_THREADS) k_cols_fwd(const float2* __restrict__ inter, int nplanes,
                                                          int rows_in, int h, int hp,
                                                          float2* __restrict__ out, int ldf,
                                                          const float2* __restrict__ tw, int* __restrict__ flag,
                                                          long long max_polls) {
  constexpr int R = P / 32;
  constexpr int KB = NC / PB;
  constexpr int LDT = col_ld<NC>();
  extern __shared__ float4 col_smem4[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(col_smem4);
  float2* s_tw = reinterpret_cast<float2*>(col_smem4 + 1);
  float2* tile = s_tw + tw_pad(P);
  const int kx0 = blockIdx.x * KB, pl0 = blockIdx.y * PB;
  const int LP = plane_ld(nplanes);
  const int kb = min(KB, h - kx0), np = min(PB, nplanes - pl0);
  if constexpr (BULK) {
    const unsigned run = (unsigned)((np + 1) & ~1) * sizeof(float2);
    if (!col_stage_in<P>(
            bar, s_tw, tw, rows_in * kb, run,
            [&](int r) { return inter + ((size_t)(r / kb) * hp + kx0 + r % kb) * LP + pl0; },
            [&](int r) { return tile + (r / kb) * LDT + (r % kb) * PB; }, flag, max_polls))
      return;
  } else {
    for (int i = threadIdx.x; i < tw_pad(P); i += COL_THREADS) s_tw[i] = tw[i];
    for (int idx = threadIdx.x; idx < rows_in * NC; idx += COL_THREADS) {
      const int row = idx / NC, cc = idx % NC;
      const int kx = kx0 + cc / PB, pl = pl0 + cc % PB;
      float2 val = make_float2(0.f, 0.f);
      if (kx < h && pl < nplanes) val = inter[((size_t)row * hp + kx) * LP + pl];
      tile[row * LDT + cc] = val;
    }
    __syncthreads();
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = 2 * warp; c < NC; c += 2 * (COL_THREADS / 32)) {
    cpair v[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int y = lane + 32 * i;
      if (y < rows_in)
        vld(v[i], tile + y * LDT + c);
      else
        vzero(v[i]);
    }
    warp_fft<P, false>(v, lane, s_tw, tile + c, LDT);
#pragma unroll
    for (int i = 0; i < R; ++i) vst(tile + col_row<P>(out_pos<P>(lane, i)) * LDT + c, v[i]);
  }
  if constexpr (BULK) {
    col_stage_out(
        P * kb, np, [&](int r) { return tile + col_row<P>(r / kb) * LDT + (r % kb) * PB; },
        [&](int r) { return out + ((size_t)(r / kb) * h + kx0 + r % kb) * ldf + pl0; });
  } else {
    __syncthreads();
    for (int idx = threadIdx.x; idx < P * NC; idx += COL_THREADS) {
      const int ky = idx / NC, cc = idx % NC;
      const int kx = kx0 + cc / PB, pl = pl0 + cc % PB;
      if (kx < h && pl < nplanes) out[((size_t)ky * h + kx) * ldf + pl] = tile[col_row<P>(ky) * LDT + cc];
    }
  }
}

// Inverse C2C along y: in[ky h + kx][ldf] -> inter[row][kx][LP] for the first rows_out rows.
template <int P, int PB, int NC, bool BULK>
__global__ void __launch_bounds__(COL_THREADS) k_cols_inv(const float2* __restrict__ in, int ldf, int nplanes,
                                                          int rows_out, int h, int hp,
                                                          float2* __restrict__ inter,
                                                          const float2* __restrict__ tw, int* __restrict__ flag,
                                                          long long max_polls) {
  constexpr int R = P / 32;
  constexpr int KB = NC / PB;
  constexpr int LDT = col_ld<NC>();
  extern __shared__ float4 col_smem4[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(col_smem4);
  float2* s_tw = reinterpret_cast<float2*>(col_smem4 + 1);
  float2* tile = s_tw + tw_pad(P);
  const int kx0 = blockIdx.x * KB, pl0 = blockIdx.y * PB;
  const int LP = plane_ld(nplanes);
  const int kb = min(KB, h - kx0), np = min(PB, nplanes - pl0);
  if constexpr (BULK) {
    // runs rounded up to an even plane count stay inside the ldf pitch (a multiple of 8)
    const unsigned run = (unsigned)((np + 1) & ~1) * sizeof(float2);
    if (!col_stage_in<P>(
            bar, s_tw, tw, P * kb, run,
            [&](int r) { return in + ((size_t)(r / kb) * h + kx0 + r % kb) * ldf + pl0; },
            [&](int r) { return tile + (r / kb) * LDT + (r % kb) * PB; }, flag, max_polls))
      return;
  } else {
    for (int i = threadIdx.x; i < tw_pad(P); i += COL_THREADS) s_tw[i] = tw[i];
    for (int idx = threadIdx.x; idx < P * NC; idx += COL_THREADS) {
      const int ky = idx / NC, cc = idx % NC;
      const int kx = kx0 + cc / PB, pl = pl0 + cc % PB;
      float2 val = make_float2(0.f, 0.f);
      if (kx < h && pl < nplanes) val = in[((size_t)ky * h + kx) * ldf + pl];
      tile[ky * LDT + cc] = val;
    }
    __syncthreads();
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = 2 * warp; c < NC; c += 2 * (COL_THREADS / 32)) {
    cpair v[R];
#pragma unroll
    for (int i = 0; i < R; ++i) vld(v[i], tile + (lane + 32 * i) * LDT + c);
    warp_fft<P, true>(v, lane, s_tw, tile + c, LDT);
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int y = out_pos<P>(lane, i);
      if (y < rows_out) vst(tile + col_row<P>(y) * LDT + c, v[i]);
    }
  }
  if constexpr (BULK) {
    col_stage_out(
        rows_out * kb, np, [&](int r) { return tile + col_row<P>(r / kb) * LDT + (r % kb) * PB; },
        [&](int r) { return inter + ((size_t)(r / kb) * hp + kx0 + r % kb) * LP + pl0; });
  } else {
    __syncthreads();
    for (int idx = threadIdx.x; idx < rows_out * NC; idx += COL_THREADS) {
      const int row = idx / NC, cc = idx % NC;
      const int kx = kx0 + cc / PB, pl = pl0 + cc % PB;
      if (kx < h && pl < nplanes) inter[((size_t)row * hp + kx) * LP + pl] = tile[col_row<P>(row) * LDT + cc];
    }
  }
}

// ------------------------------------------------------------ launchers ----

size_t row_smem(int p) {
  return (size_t)(tw_pad(p) + (p / 2 + 1) * SH_LD + ROW_WARPS * (p + 2)) * sizeof(float2);
}

// Bulk staging needs 16-byte aligned buffers and an even spectrum pitch (the
// intermediate's plane pitch is a multiple of 16).
bool cols_bulk_ok(const void* a, const void* b, const void* tw, int ldf) {
  return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(tw)) &
          15) == 0 &&
         (ldf & 1) == 0;
}

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

// Tile codes: PB for NC = 32 (8, 16, 32), 100 + PB for NC = 16 (108, 116);
// code 0 = the element-wise variant (NC = 32, PB = 8) for buffers the bulk
// copies cannot take.
#define CTOF_COLS_CASE(KERN, PB_, NC_, BULK_, ...)                       \
  CTOF_P_SWITCH(k->p, {                                                  \
    CTOF_CUDA_TRY(allow_smem(KERN<P_, PB_, NC_, BULK_>, sm));            \
    KERN<P_, PB_, NC_, BULK_><<<grid, COL_THREADS, sm, st>>>(__VA_ARGS__); \
  })

#define CTOF_COLS_LAUNCH(KERN, ...)                                                         \
  do {                                                                                      \
    const int pb = code == 0 ? 8 : (code >= 100 ? code - 100 : code), nc = code >= 100 ? 16 : 32; \
    const size_t sm = col_smem_bytes(k->p, nc);                                             \
    dim3 grid(ctof_div_up(k->h, nc / pb), ctof_div_up(nplanes, pb));                       \
    switch (code) {                                                                         \
      case 0: CTOF_COLS_CASE(KERN, 8, 32, false, __VA_ARGS__); break;                       \
      case 32: CTOF_COLS_CASE(KERN, 32, 32, true, __VA_ARGS__); break;                      \
      case 16: CTOF_COLS_CASE(KERN, 16, 32, true, __VA_ARGS__); break;                      \
      case 116: CTOF_COLS_CASE(KERN, 16, 16, true, __VA_ARGS__); break;                     \
      case 108: CTOF_COLS_CASE(KERN, 8, 16, true, __VA_ARGS__); break;                      \
      default: CTOF_COLS_CASE(KERN, 8, 32, true, __VA_ARGS__);                              \
    }                                                                                       \
  } while (0)

ctof_status fft_cols_forward_pb(const ctof_kernel_s* k, const float2* inter, int nplanes, int rows_in, float2* out,
                                int ldf, int code, cudaStream_t st) {
  if (nplanes <= 0) return CTOF_OK;
  if (!cols_bulk_ok(inter, out, k->d_tw, ldf)) code = 0;
  CTOF_COLS_LAUNCH(k_cols_fwd, inter, nplanes, rows_in, k->h, k->hp, out, ldf, k->d_tw, k->d_flags, k->max_polls);
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
  if (!cols_bulk_ok(in, inter, k->d_tw, ldf)) code = 0;
  CTOF_COLS_LAUNCH(k_cols_inv, in, ldf, nplanes, rows_out, k->h, k->hp, inter, k->d_tw, k->d_flags, k->max_polls);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status fft_cols_inverse(const ctof_kernel_s* k, const float2* in, int ldf, int nplanes, int rows_out,
                             float2* inter, cudaStream_t st) {
  const int pb = (nplanes == k->nt) ? k->tune_pb[1] : k->tune_pb[3];
  return fft_cols_inverse_pb(k, in, ldf, nplanes, rows_out, inter, pb, st);
}

int fft_twiddle_count(int p) { return tw_pad(p); }

void fft_twiddle_table(int p, float2* out) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int i = 0; i < tw_pad(p); ++i) {
    int j = 0;
    if (i < p) {
      j = i;
    } else if (i < p + 31) {
      const int e = i - p;
      int s = 1;
      while (2 * s - 1 <= e) s *= 2;  // stage s holds entries s-1 .. 2s-2
      j = (e - (s - 1)) * (p / (2 * s));
    } else if (i < tw_count(p)) {
      const int e = i - p - 31;
      j = ((e & 31) * (e / 32 + 1)) & (p - 1);
    }
    out[i] = make_float2((float)cos(two_pi * j / p), (float)-sin(two_pi * j / p));
  }
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
