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
//           planes at a time (persistent over jobs); each warp transforms the
//           rows of two planes packed as one complex row and splits them with
//           the Hermitian identities; the 16 planes' half spectra of the row
//           move between the intermediate and shared memory as tensor-map
//           boxes (16 planes x up to 256 kx), double-buffered so that the next
//           job's box is in flight while the CTA works on the current one.
//   columns (y axis, complex): a CTA holds NC columns (NC/PB kx x PB
//           consecutive planes, PB = 8 or 16, NC = 16 or 32, picked per handle
//           by the autotuner) of all rows, loaded and stored as tensor-map
//           boxes (PB planes x 1 kx x up to 256 rows); each warp transforms two
//           columns at once.  The transpose between plane-major input planes
//           and frequency-major spectra happens in the row pass.
// Shared-memory tiles use the copy engine's 64/128-byte swizzle, under which
// the 16-byte accesses of a quarter-warp to eight rows that are distinct mod 8
// are conflict-free; out-of-range planes, kx and rows are zero-filled by the
// loads and skipped by the stores.
// Each 1-D transform of length P = 32 R lives in one warp: lane l register i
// holds element l + 32 i; an R-point DFT over the registers (constant
// twiddles), a twiddle by w_P^(l k1), and a 32-point DFT across the lanes,
// from P = 256 on as 4 x 8 points in registers through the warp's scratch,
// below as five shuffle stages.  Twiddles are computed on the host in double
// precision and staged in shared memory.
#include <cuda_runtime.h>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include "bulk.cuh"
#include "ctof_internal.h"

namespace {

// Column-pass tiles hold NC = 32 or 16 columns: KB kx-columns x PB planes;
// the tile shape (NC, PB) is chosen per handle and use by the autotuner
// (tile code PB for NC = 32, 100 + PB for NC = 16).
constexpr int COL_THREADS = 256;
constexpr int ROW_WARPS = 8;

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }

__device__ __forceinline__ int brev5(int l) { return (int)(__brev((unsigned)l) >> 27); }

// Twiddle table, built on the host in this layout and copied to shared memory
// as is: the P roots w^j, then copies of the values that the lanes need at
// the same time, so that those reads hit distinct banks:
// [P + s - 1 + l] = w^(l P / 2s) for the cross-lane stage s (l < s),
// [P + 31 + 32 (k - 1) + lane] = w^(lane k) for the register twiddles, and
// [tw4_base(P) + 8 (m1 - 1) + b] = w^(R b m1) for the 4 x 8 step (m1 = 1..3,
// b < 8); padded to an even count (a multiple of 16 bytes).
__host__ __device__ constexpr int tw4_base(int P) { return P + 31 + 32 * (P / 32 - 1); }
__host__ __device__ constexpr int tw_count(int P) { return tw4_base(P) + 24; }
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
__device__ __forceinline__ void vst(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void vld(cpair& v, const float2* p) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v.a = make_float2(q.x, q.y);
  v.b = make_float2(q.z, q.w);
}
__device__ __forceinline__ void vst(float2* p, cpair v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.a.x, v.a.y, v.b.x, v.b.y);
}
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
// [0, P)): S[i][l] (register i, lane l) and S2[i][m1][b].  Column tiles
// (16-byte accesses, swizzled rows): eight consecutive lanes touch eight
// slots that are distinct mod 8.  Row buffers (8-byte accesses, unit stride):
// sixteen consecutive lanes touch sixteen slots that are distinct mod 16.
__device__ __forceinline__ int slot_a(int i, int l) { return i * 32 + ((l + 8 * (i & 1)) & 31); }
__device__ __forceinline__ int slot_c_tile(int i, int m1, int b) { return (4 * i + m1) * 8 + (b ^ (i & 7)); }
__device__ __forceinline__ int slot_c_row(int i, int m1, int b) {
  const int t = 4 * i + m1;
  return (t >> 4) * 128 + b * 16 + ((t & 15) ^ ((b & 3) | ((b & 4) << 1)));
}

// Where a warp transform keeps its intermediate values: FFT_SHFL (five
// shuffle stages), FFT_TILE (a column pair of the column-pass tile) or
// FFT_ROWBUF (the warp's own row buffer); the last two run the 4 x 8 step
// when P >= 256 and the shuffles otherwise.  They differ in which lanes
// finish which outputs: FFT_TILE gives eight consecutive lanes eight k1
// values that are distinct mod 8 (outputs go to natural tile rows),
// FFT_ROWBUF four k1 x four k2 per half-warp.
constexpr int FFT_SHFL = 0, FFT_TILE = 1, FFT_ROWBUF = 2;

// Length-P DFT held by one warp, P = 32 R: lane l register i holds element
// l + 32 i (of one column, or of each of two columns).  X[k1 + R k2] =
// sum_l w32^(l k2) w_P^(l k1) sum_i x[l + 32 i] w_R^(i k1): an R-point DFT
// over the registers (register i then holds k1 = i), the twiddle w_P^(l k1),
// and a 32-point DFT across the lanes.  INV selects exp(+...).
// With a scratch MODE and P >= 256 the 32-point DFT across the lanes runs as
// 4 x 8 points in registers with two passes through the scratch (scr(s) is
// the address of slot s, s < P):
//   Z[m1 + 4 m2] = sum_b w8^(b m2) w32^(b m1) sum_a y[b + 8 a] w4^(a m1);
// otherwise as five shuffle stages (DIF, outputs in bit-reversed lane order).
template <int P, bool INV, int MODE, typename T, typename Scr>
__device__ __forceinline__ void warp_fft(T (&v)[P / 32], int lane, const float2* tw, const Scr& scr) {
  constexpr int R = P / 32;
  reg_dft<R, INV>(v);
#pragma unroll
  for (int i = 1; i < R; ++i) v[i] = vmul(v[i], tw_conj<INV>(tw[P + 31 + 32 * (i - 1) + lane]));
  if constexpr (MODE != FFT_SHFL && R >= 8) {
    __syncwarp();  // every lane has read its inputs (callers may pass their input column as scratch)
#pragma unroll
    for (int i = 0; i < R; ++i) vst(scr(slot_a(i, lane)), v[i]);
    __syncwarp();
    const int b = lane & 7;
    T t[R / 4][4];
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
      const int i = (lane >> 3) + 4 * q;
#pragma unroll
      for (int a = 0; a < 4; ++a) vld(t[q][a], scr(slot_a(i, b + 8 * a)));
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
      const int i = (lane >> 3) + 4 * q;
      dft4<INV>(t[q][0], t[q][1], t[q][2], t[q][3]);
#pragma unroll
      for (int m1 = 1; m1 < 4; ++m1) t[q][m1] = vmul(t[q][m1], tw_conj<INV>(tw[tw4_base(P) + 8 * (m1 - 1) + b]));
#pragma unroll
      for (int m1 = 0; m1 < 4; ++m1) {
        const int s = MODE == FFT_TILE ? slot_c_tile(i, m1, b) : slot_c_row(i, m1, b);
        vst(scr(s), t[q][m1]);
      }
    }
    __syncwarp();
    const int m1 = MODE == FFT_TILE ? lane >> 3 : lane & 3;
#pragma unroll
    for (int q = 0; q < R / 8; ++q) {
      const int i = (MODE == FFT_TILE ? (lane & 7) : (lane >> 2)) + 8 * q;
      T u[8];
#pragma unroll
      for (int bb = 0; bb < 8; ++bb)
        vld(u[bb], scr(MODE == FFT_TILE ? slot_c_tile(i, m1, bb) : slot_c_row(i, m1, bb)));
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

// Output position of register i of lane `lane` after warp_fft<P, INV, MODE>.
template <int P, int MODE>
__device__ __forceinline__ int out_pos(int lane, int i) {
  constexpr int R = P / 32;
  if constexpr (MODE == FFT_TILE && R >= 8) {
    // register 8 q + m2 of lane L: k1 = (L & 7) + 8 q, k2 = (L >> 3) + 4 m2
    return (lane & 7) + 8 * (i >> 3) + R * ((lane >> 3) + 4 * (i & 7));
  } else if constexpr (MODE == FFT_ROWBUF && R >= 8) {
    // register 8 q + m2 of lane L: k1 = (L >> 2) + 8 q, k2 = (L & 3) + 4 m2
    return (lane >> 2) + 8 * (i >> 3) + R * ((lane & 3) + 4 * (i & 7));
  } else {
    return i + R * brev5(lane);
  }
}

// Unit-stride scratch (a warp's row buffer).
struct LinearScr {
  float2* p;
  __device__ __forceinline__ float2* operator()(int s) const { return p + s; }
};

// ---------------------------------------------------------------- rows ----

constexpr int RP = 2 * ROW_WARPS;  // planes per row-pass CTA

__host__ __device__ inline int plane_ld(int nplanes) { return (nplanes + RP - 1) / RP * RP; }

// Half spectra of the CTA's planes for one row: s_h[kx][plane], 16 planes =
// 128 bytes per kx, in the TMA 128-byte swizzle (the 16-byte chunk of planes
// 2c, 2c + 1 of row s sits at chunk c ^ (s & 7)), so that a warp's plane pair
// is one conflict-free 16-byte access for consecutive kx.  Loaded and stored
// as boxes of RKX(P) kx; for P = 512 the second box starts at s_h row
// RKX_GAP(P) (1024-byte aligned).  Two buffers: the copies of the next job
// land in one while the CTA works on the other.
__host__ __device__ constexpr int rkx(int P) { return P / 2 + 1 <= 256 ? P / 2 + 1 : P / 4 + 1; }
__host__ __device__ constexpr int rkx_boxes(int P) { return P / 2 + 1 <= 256 ? 1 : 2; }
__host__ __device__ constexpr int rkx_second(int P) { return (rkx(P) + 7) / 8 * 8; }  // s_h row of box 2
__host__ __device__ constexpr int sh_rows(int P) { return rkx_boxes(P) == 1 ? rkx(P) : rkx_second(P) + rkx(P); }
__host__ __device__ constexpr int sh_bytes(int P) { return (sh_rows(P) * 128 + 1023) / 1024 * 1024; }

template <int P>
__device__ __forceinline__ int sh_row(int kx) {
  if constexpr (rkx_boxes(P) == 1) {
    return kx;
  } else {
    return kx < rkx(P) ? kx : kx - rkx(P) + rkx_second(P);
  }
}

// Address of the plane pair (2 c, 2 c + 1) of kx in an s_h buffer.
template <int P>
__device__ __forceinline__ float2* sh_at(float2* s_h, int kx, int c) {
  const int s = sh_row<P>(kx);
  return s_h + s * 16 + ((c ^ (s & 7)) << 1);
}

// The row transforms run the 4 x 8 step in the warp's buffer from P = 256 on.
template <int P>
__host__ __device__ constexpr int row_mode() {
  return P >= 256 ? FFT_ROWBUF : FFT_SHFL;
}

// Row-buffer slot of transform output e: a permutation of [0, P) under which
// the sixteen outputs that a half-warp writes with one register, and sixteen
// consecutive outputs, fall on distinct 8-byte banks (4 x 8 path: XOR of
// bits 2-3 with bits log2 R .. log2 R + 1; shuffle path: the low log2 R bits
// with the next ones).
template <int P>
__device__ __forceinline__ int row_pos(int e) {
  constexpr int R = P / 32;
  if constexpr (row_mode<P>() == FFT_ROWBUF) {
    return e ^ (((e / R) & 3) << 2);
  } else {
    return e ^ ((e / R) & (R - 1));
  }
}

// Row-pass shared memory (from a 1024-byte aligned base):
// [s_h x 2][twiddles][per-warp buffers of P + 2][2 mbarriers].
__host__ __device__ constexpr size_t row_smem_bytes(int P) {
  return 1024 + 2 * (size_t)sh_bytes(P) + ((size_t)tw_pad(P) + (size_t)ROW_WARPS * (P + 2)) * sizeof(float2) + 16;
}

struct RowSmem {
  float2* s_h;  // buffer b at s_h + b * sh_bytes / 8
  float2* s_tw;
  float2* buf;
  uint64_t* bar;
};

__device__ __forceinline__ char* align1024(void* p) {
  const uint32_t s = bulk::saddr(p);
  return static_cast<char*>(p) + (((s + 1023u) & ~1023u) - s);
}

template <int P>
__device__ __forceinline__ RowSmem row_carve(float4* raw, int warp) {
  RowSmem m;
  char* base = align1024(raw);
  m.s_h = reinterpret_cast<float2*>(base);
  m.s_tw = reinterpret_cast<float2*>(base + 2 * sh_bytes(P));
  float2* bufs = m.s_tw + tw_pad(P);
  m.buf = bufs + warp * (P + 2);
  m.bar = reinterpret_cast<uint64_t*>(bufs + ROW_WARPS * (P + 2));
  return m;
}

template <int P>
__device__ __forceinline__ float2* sh_buf(const RowSmem& S, int b) {
  return S.s_h + b * (sh_bytes(P) / (int)sizeof(float2));
}

// Block-wide prologue: barriers (one per s_h buffer) and twiddles.
template <int P>
__device__ __forceinline__ void row_prologue(const RowSmem& S, const float2* tw) {
  if (threadIdx.x == 0) {
    bulk::bar_init(S.bar, 1);
    bulk::bar_init(S.bar + 1, 1);
  }
  for (int i = threadIdx.x; i < tw_pad(P); i += blockDim.x) S.s_tw[i] = tw[i];
  __syncthreads();  // barriers initialised and twiddles staged before any use
}

// Block-wide wait for the copies into buffer (it & 1) of iteration `it`
// (phase it / 2 of that buffer's barrier); false, with the handle's status
// flag set, when they did not land within max_polls polls.
__device__ __forceinline__ bool row_wait(uint64_t* bar, int it, int* flag, long long max_polls) {
  const uint32_t parity = (uint32_t)(it >> 1) & 1u;
  const bool ok = bulk::block_wait(bar, parity, max_polls);
  if (!ok && threadIdx.x == 0) {
    atomicOr(flag, 1);
    bulk::wait(bar, parity, bulk::DRAIN_POLLS);
  }
  return ok;
}

// One thread: row r, planes pl0.. of the intermediate into buffer s_h as
// rkx_boxes tensor copies, completing on bar.
template <int P>
__device__ __forceinline__ void row_load_issue(uint64_t* bar, float2* s_h, const CUtensorMap* map, int r, int pl0) {
  bulk::arrive_expect(bar, rkx_boxes(P) * rkx(P) * 128u);
  bulk::tensor_g2s(s_h, map, pl0, 0, r, bar);
  if constexpr (rkx_boxes(P) == 2) bulk::tensor_g2s(s_h + rkx_second(P) * 16, map, pl0, rkx(P), r, bar);
}

// Block-wide: buffer s_h back to row r of the intermediate (one thread issues
// the tensor copies into its bulk group); planes past the last and kx past h
// are skipped by the copy.
template <int P>
__device__ __forceinline__ void row_store(const float2* s_h, const CUtensorMap* map, int r, int pl0) {
  bulk::fence_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    bulk::tensor_s2g(map, pl0, 0, r, s_h);
    if constexpr (rkx_boxes(P) == 2) bulk::tensor_s2g(map, pl0, rkx(P), r, s_h + rkx_second(P) * 16);
    bulk::commit();
  }
}

template <int P>
__device__ __forceinline__ void split_to_tile(const float2* buf, int lane, float2* s_h, int c) {
  for (int kk = lane; kk <= P / 2; kk += 32) {
    const float2 zk = buf[row_pos<P>(kk)];
    const float2 zm = buf[row_pos<P>((P - kk) & (P - 1))];
    *reinterpret_cast<float4*>(sh_at<P>(s_h, kk, c)) =
        make_float4(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y), 0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
  }
}

// Z[n] = A[n] + i B[n] from the half spectra of plane pair c (zero for planes
// past the last: has0 / has1 false).
template <int P>
__device__ __forceinline__ void load_pair_from_tile(float2 (&v)[P / 32], float2* s_h, int c, int lane, bool has0,
                                                    bool has1) {
  constexpr int R = P / 32;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int n = lane + 32 * i;
    float4 q = *reinterpret_cast<const float4*>(sh_at<P>(s_h, n <= P / 2 ? n : P - n, c));
    if (n > P / 2) {
      q.y = -q.y;
      q.w = -q.w;
    }
    if (!has0) q.x = q.y = 0.f;
    if (!has1) q.z = q.w = 0.f;
    v[i] = make_float2(q.x - q.w, q.y + q.z);
  }
}

// One warp transform of a packed row pair, results left in the warp's buffer
// at row_pos slots.
template <int P, bool INV>
__device__ __forceinline__ void row_transform(float2 (&v)[P / 32], int lane, const RowSmem& S) {
  constexpr int R = P / 32;
  warp_fft<P, INV, row_mode<P>()>(v, lane, S.s_tw, LinearScr{S.buf});
#pragma unroll
  for (int i = 0; i < R; ++i) S.buf[row_pos<P>(out_pos<P, row_mode<P>()>(lane, i))] = v[i];
  __syncwarp();
}

// Forward R2C of rows: in[plane][row][ld_in] (first cols_in columns, zero beyond)
// -> inter[row][kx][plane] (tensor map `dst`: nplanes x h x rows).
template <int P>
__global__ void __launch_bounds__(ROW_WARPS * 32) k_rows_fwd(const __grid_constant__ CUtensorMap dst,
                                                             const float* __restrict__ in, int nplanes, int rows,
                                                             int cols_in, int ld_in, const float2* __restrict__ tw) {
  constexpr int R = P / 32;
  extern __shared__ float4 row_smem4[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const RowSmem S = row_carve<P>(row_smem4, warp);
  row_prologue<P>(S, tw);
  const int nblk = plane_ld(nplanes) / RP;
  int it = 0;
  for (int job = blockIdx.x; job < rows * nblk; job += gridDim.x, ++it) {
    const int r = job / nblk, pl0 = (job - r * nblk) * RP;
    const int p0 = pl0 + 2 * warp, p1 = p0 + 1;
    float2* s_h = sh_buf<P>(S, it & 1);
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
    row_transform<P, false>(v, lane, S);
    if (threadIdx.x == 0) bulk::wait_read<1>();  // the copy out of this buffer two jobs ago has read it
    __syncthreads();
    split_to_tile<P>(S.buf, lane, s_h, warp);
    row_store<P>(s_h, &dst, r, pl0);
  }
  if (threadIdx.x == 0) bulk::wait_read<0>();
}

// Inverse C2R of rows: inter[row][kx][plane] (tensor map `src`) ->
// out[plane][row][ld_out] (first cols_out columns), x scale.  With NORM
// nothing is stored: `out` is read as a reference y of the same layout and
// the block adds sum (scale z - y)^2 and sum y^2 over the kept columns to
// acc[0] and acc[1].
template <int P, bool NORM>
__global__ void __launch_bounds__(ROW_WARPS * 32) k_rows_inv(const __grid_constant__ CUtensorMap src, int nplanes,
                                                             int rows, int cols_out, float* __restrict__ out,
                                                             int ld_out, float scale,
                                                             const float2* __restrict__ tw, int* __restrict__ flag,
                                                             long long max_polls, double* __restrict__ acc) {
  constexpr int R = P / 32;
  extern __shared__ float4 row_smem4[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const RowSmem S = row_carve<P>(row_smem4, warp);
  row_prologue<P>(S, tw);
  const int nblk = plane_ld(nplanes) / RP, njobs = rows * nblk;
  auto issue = [&](int job, int it) {
    const int r = job / nblk;
    row_load_issue<P>(S.bar + (it & 1), sh_buf<P>(S, it & 1), &src, r, (job - r * nblk) * RP);
  };
  float sr = 0.f, sy = 0.f;  // NORM partial sums of this lane
  if (threadIdx.x == 0 && (int)blockIdx.x < njobs) issue(blockIdx.x, 0);
  int it = 0;
  for (int job = blockIdx.x; job < njobs; job += gridDim.x, ++it) {
    const int r = job / nblk, pl0 = (job - r * nblk) * RP;
    const int p0 = pl0 + 2 * warp, p1 = p0 + 1;
    // the other buffer was last read in the previous iteration, before its closing barrier
    if (threadIdx.x == 0 && job + (int)gridDim.x < njobs) issue(job + gridDim.x, it + 1);
    if (!row_wait(S.bar + (it & 1), it, flag, max_polls)) {
      if (threadIdx.x == 0 && job + (int)gridDim.x < njobs)  // the next job's copies are in flight too
        bulk::wait(S.bar + ((it + 1) & 1), (uint32_t)((it + 1) >> 1) & 1u, bulk::DRAIN_POLLS);
      return;
    }
    float2 v[R];
    load_pair_from_tile<P>(v, sh_buf<P>(S, it & 1), warp, lane, p0 < nplanes, p1 < nplanes);
    row_transform<P, true>(v, lane, S);
    for (int c = lane; c < cols_out; c += 32) {
      const float2 z = S.buf[row_pos<P>(c)];
      const size_t o0 = ((size_t)p0 * rows + r) * ld_out + c, o1 = ((size_t)p1 * rows + r) * ld_out + c;
      if constexpr (NORM) {
        if (p0 < nplanes) {
          const float y = out[o0], d = z.x * scale - y;
          sr = fmaf(d, d, sr);
          sy = fmaf(y, y, sy);
        }
        if (p1 < nplanes) {
          const float y = out[o1], d = z.y * scale - y;
          sr = fmaf(d, d, sr);
          sy = fmaf(y, y, sy);
        }
      } else {
        if (p0 < nplanes) out[o0] = z.x * scale;
        if (p1 < nplanes) out[o1] = z.y * scale;
      }
    }
    bulk::fence_smem();  // this job's reads of its buffer, before later copies overwrite it
    __syncthreads();
  }
  if constexpr (NORM) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) {
      atomicAdd(acc, (double)sr);
      atomicAdd(acc + 1, (double)sy);
    }
  }
}

// ADMM T side, per measurement row y and pair of time bins t:
//   Kx   = C2R(row spectra) on the N scan columns
//   a1   = Kx + u1;  v1 = (m/scale + rho a1) / (1 + rho);  u1 <- a1 - v1
//   c    = (v1 - u1) - Kx = 2 v1 - a1 - Kx      (zero off the scan)
//   row spectra <- R2C(c zero-padded to P)
// so that FFT(v1 - u1) = K x_hat + c_hat without a transform of the full
// P x P plane.  With RESID the update is the data residual of the gradient
// A^T (A x - m) instead: c = Kx - m on the scan (Kx alone when m is null;
// u1, inv_s and rho unused).  m, u1: [nt][n][n]; inter: [n][kx][plane] in
// place (tensor map `map`).  The m and u1 values of a lane are loaded before
// its tile is waited for; the next job's tile is requested once the copy out
// of its buffer has read it.
template <int P, bool RESID>
__global__ void __launch_bounds__(ROW_WARPS * 32, P >= 512 ? 2 : 3)
    k_rows_admm_t(const __grid_constant__ CUtensorMap map, int nplanes, int n, const float* __restrict__ m,
                  float* __restrict__ u1, float scale, float inv_s, float rho, const float2* __restrict__ tw,
                  int* __restrict__ flag, long long max_polls) {
  constexpr int R = P / 32;
  constexpr int RN = R / 2 > 0 ? R / 2 : 1;  // registers that can hold scan columns (n <= P / 2)
  extern __shared__ float4 row_smem4[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const RowSmem S = row_carve<P>(row_smem4, warp);
  row_prologue<P>(S, tw);
  const float inv1r = 1.0f / (1.0f + rho);
  const int nblk = plane_ld(nplanes) / RP, njobs = n * nblk;
  auto issue = [&](int job, int it) {
    const int r = job / nblk;
    row_load_issue<P>(S.bar + (it & 1), sh_buf<P>(S, it & 1), &map, r, (job - r * nblk) * RP);
  };
  if (threadIdx.x == 0 && (int)blockIdx.x < njobs) issue(blockIdx.x, 0);
  int it = 0;
  for (int job = blockIdx.x; job < njobs; job += gridDim.x, ++it) {
    const int r = job / nblk, pl0 = (job - r * nblk) * RP;
    const int p0 = pl0 + 2 * warp, p1 = p0 + 1;
    const bool has0 = p0 < nplanes, has1 = p1 < nplanes;
    float2* s_h = sh_buf<P>(S, it & 1);
    float mv0[RN], mv1[RN], uv0[RN], uv1[RN];
    const size_t row0 = ((size_t)p0 * n + r) * n, row1 = ((size_t)p1 * n + r) * n;
#pragma unroll
    for (int i = 0; i < RN; ++i) {
      const int c = lane + 32 * i;
      mv0[i] = uv0[i] = mv1[i] = uv1[i] = 0.f;
      if constexpr (RESID) {
        if (m != nullptr && c < n) {
          if (has0) mv0[i] = m[row0 + c];
          if (has1) mv1[i] = m[row1 + c];
        }
      } else {
        if (c < n && has0) {
          mv0[i] = m[row0 + c];
          uv0[i] = u1[row0 + c];
        }
        if (c < n && has1) {
          mv1[i] = m[row1 + c];
          uv1[i] = u1[row1 + c];
        }
      }
    }
    if (!row_wait(S.bar + (it & 1), it, flag, max_polls)) {
      if (threadIdx.x == 0) bulk::wait_read<0>();  // the previous job's copy out of shared memory
      return;
    }
    float2 v[R];
    load_pair_from_tile<P>(v, s_h, warp, lane, has0, has1);
    row_transform<P, true>(v, lane, S);
    if (threadIdx.x == 0) {
      bulk::wait_read<0>();  // the previous job's copy has read the other buffer
      if (job + (int)gridDim.x < njobs) issue(job + gridDim.x, it + 1);
    }
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < RN; ++i) {
      const int c = lane + 32 * i;
      if (c < n) {
        const float2 kx = cscale(S.buf[row_pos<P>(c)], scale);
        if constexpr (RESID) {
          if (has0) v[i].x = kx.x - mv0[i];
          if (has1) v[i].y = kx.y - mv1[i];
          continue;
        }
        if (has0) {
          const float a1 = kx.x + uv0[i];
          const float v1 = (mv0[i] * inv_s + rho * a1) * inv1r;
          u1[row0 + c] = a1 - v1;
          v[i].x = 2.f * v1 - a1 - kx.x;
        }
        if (has1) {
          const float a1 = kx.y + uv1[i];
          const float v1 = (mv1[i] * inv_s + rho * a1) * inv1r;
          u1[row1 + c] = a1 - v1;
          v[i].y = 2.f * v1 - a1 - kx.y;
        }
      }
    }
    __syncwarp();
    row_transform<P, false>(v, lane, S);
    __syncthreads();  // every warp is done reading this job's buffer
    split_to_tile<P>(S.buf, lane, s_h, warp);
    row_store<P>(s_h, &map, r, pl0);
  }
  if (threadIdx.x == 0) bulk::wait_read<0>();
}

// ------------------------------------------------------------- columns ----

// Column-pass tile: NC columns = KB kx-columns x PB consecutive planes, all
// P rows; kx-column j is a region [row][PB planes] loaded and stored as
// tensor boxes of RB = min(P, 256) rows, in the TMA swizzle of its row size
// (PB = 16: 128-byte rows, the 16-byte chunk c of row r at c ^ (r & 7);
// PB = 8: 64-byte rows, chunk c at c ^ ((r >> 1) & 3)), so that eight rows
// that are distinct mod 8 put a quarter-warp's 16-byte accesses on distinct
// bank groups.  Each warp transforms two adjacent columns at once (cpair).
template <int P>
__host__ __device__ constexpr int col_rb() {
  return P < 256 ? P : 256;
}

template <int PB>
struct ColPair {
  float2* region;  // the kx-column's region
  int c;           // the pair's 16-byte chunk within a row
  __device__ __forceinline__ float2* operator()(int r) const {
    if constexpr (PB == 16) {
      return region + r * 16 + ((c ^ (r & 7)) << 1);
    } else {
      return region + r * 8 + ((c ^ ((r >> 1) & 3)) << 1);
    }
  }
};

// Shared memory of a column pass (from a 1024-byte aligned base): [tile][twiddles][mbarrier].
__host__ __device__ constexpr size_t col_smem_bytes(int P, int NC) {
  return 1024 + ((size_t)P * NC + (size_t)tw_pad(P)) * sizeof(float2) + 16;
}

// One thread: the twiddles and the tile's boxes (kx-columns j < kb, row boxes
// rb < nrb of map `src` at planes pl0, kx0 + j, rows rb RB) into shared memory,
// completing on bar.
template <int P, int PB>
__device__ __forceinline__ void col_load_issue(uint64_t* bar, float2* tile, float2* s_tw, const float2* tw,
                                               const CUtensorMap* src, int pl0, int kx0, int kb, int nrb) {
  constexpr int RB = col_rb<P>();
  bulk::bar_init(bar, 1);
  bulk::arrive_expect(bar, (unsigned)(kb * nrb * RB * PB) * (unsigned)sizeof(float2) +
                               tw_pad(P) * (unsigned)sizeof(float2));
  bulk::g2s(s_tw, tw, tw_pad(P) * sizeof(float2), bar);
  for (int j = 0; j < kb; ++j)
    for (int rb = 0; rb < nrb; ++rb) bulk::tensor_g2s(tile + (j * P + rb * RB) * PB, src, pl0, kx0 + j, rb * RB, bar);
}

// Block-wide wait for col_load_issue's copies; false (status flag set) on timeout.
__device__ __forceinline__ bool col_wait(uint64_t* bar, int* flag, long long max_polls) {
  const bool ok = bulk::block_wait(bar, 0, max_polls);
  if (!ok && threadIdx.x == 0) {
    atomicOr(flag, 1);
    bulk::wait(bar, 0, bulk::DRAIN_POLLS);
  }
  return ok;
}

// Block-wide: the tile's boxes (kx-columns j < kb, row boxes rb < nrb) to map
// `dst` at planes pl0, kx0 + j, rows rb RB; one thread issues and waits until
// the copies have read shared memory.
template <int P, int PB>
__device__ __forceinline__ void col_store(const float2* tile, const CUtensorMap* dst, int pl0, int kx0, int kb,
                                          int nrb) {
  constexpr int RB = col_rb<P>();
  bulk::fence_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = 0; j < kb; ++j)
      for (int rb = 0; rb < nrb; ++rb) bulk::tensor_s2g(dst, pl0, kx0 + j, rb * RB, tile + (j * P + rb * RB) * PB);
    bulk::commit();
    bulk::wait_read<0>();
  }
}

// Forward C2C along y: inter[row][kx][plane] (map `src`: nplanes x h x
// rows_in, zero beyond) -> spectra [ky][kx][plane] (map `dst`: nplanes x h x P).
template <int P, int PB, int NC>
__global__ void __launch_bounds__(COL_THREADS) k_cols_fwd(const __grid_constant__ CUtensorMap src,
                                                          const __grid_constant__ CUtensorMap dst, int rows_in,
                                                          int h, const float2* __restrict__ tw,
                                                          int* __restrict__ flag, long long max_polls) {
  constexpr int R = P / 32;
  constexpr int KB = NC / PB;
  constexpr int RB = col_rb<P>();
  extern __shared__ float4 col_smem4[];
  float2* tile = reinterpret_cast<float2*>(align1024(col_smem4));
  float2* s_tw = tile + P * NC;
  uint64_t* bar = reinterpret_cast<uint64_t*>(s_tw + tw_pad(P));
  const int kx0 = blockIdx.x * KB, pl0 = blockIdx.y * PB;
  const int kb = min(KB, h - kx0);
  if (threadIdx.x == 0) col_load_issue<P, PB>(bar, tile, s_tw, tw, &src, pl0, kx0, kb, (rows_in + RB - 1) / RB);
  if (!col_wait(bar, flag, max_polls)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = 2 * warp; c < NC; c += 2 * (COL_THREADS / 32)) {
    const ColPair<PB> A{tile + (c / PB) * P * PB, (c % PB) >> 1};
    cpair v[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int y = lane + 32 * i;
      if (y < rows_in)
        vld(v[i], A(y));
      else
        vzero(v[i]);
    }
    warp_fft<P, false, FFT_TILE>(v, lane, s_tw, A);
#pragma unroll
    for (int i = 0; i < R; ++i) vst(A(out_pos<P, FFT_TILE>(lane, i)), v[i]);
  }
  col_store<P, PB>(tile, &dst, pl0, kx0, kb, P / RB);
}

// Inverse C2C along y: spectra [ky][kx][plane] (map `src`: nplanes x h x P) ->
// inter[row][kx][plane] for the first rows_out rows (map `dst`: nplanes x h x rows_out).
template <int P, int PB, int NC>
__global__ void __launch_bounds__(COL_THREADS) k_cols_inv(const __grid_constant__ CUtensorMap src,
                                                          const __grid_constant__ CUtensorMap dst, int rows_out,
                                                          int h, const float2* __restrict__ tw,
                                                          int* __restrict__ flag, long long max_polls) {
  constexpr int R = P / 32;
  constexpr int KB = NC / PB;
  constexpr int RB = col_rb<P>();
  extern __shared__ float4 col_smem4[];
  float2* tile = reinterpret_cast<float2*>(align1024(col_smem4));
  float2* s_tw = tile + P * NC;
  uint64_t* bar = reinterpret_cast<uint64_t*>(s_tw + tw_pad(P));
  const int kx0 = blockIdx.x * KB, pl0 = blockIdx.y * PB;
  const int kb = min(KB, h - kx0);
  if (threadIdx.x == 0) col_load_issue<P, PB>(bar, tile, s_tw, tw, &src, pl0, kx0, kb, P / RB);
  if (!col_wait(bar, flag, max_polls)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = 2 * warp; c < NC; c += 2 * (COL_THREADS / 32)) {
    const ColPair<PB> A{tile + (c / PB) * P * PB, (c % PB) >> 1};
    cpair v[R];
#pragma unroll
    for (int i = 0; i < R; ++i) vld(v[i], A(lane + 32 * i));
    warp_fft<P, true, FFT_TILE>(v, lane, s_tw, A);
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int y = out_pos<P, FFT_TILE>(lane, i);
      if (y < rows_out) vst(A(y), v[i]);
    }
  }
  col_store<P, PB>(tile, &dst, pl0, kx0, kb, (rows_out + RB - 1) / RB);
}

// ------------------------------------------------------------ launchers ----

template <typename F>
cudaError_t allow_smem(F* fn, size_t bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

int row_grid(int rows, int nplanes) {
  const int jobs = rows * (plane_ld(nplanes) / RP);
  const int cap = 152 * 8;
  return jobs < 1 ? 1 : (jobs > cap ? cap : jobs);
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// 3-D tensor map over 8-byte elements (a float2 each): planes (contiguous,
// nplanes of them), kx (h, pitch ld_kx elements), rows (pitch ld_row
// elements); box {b0, b1, b2}; swizzle = the box's inner size in bytes (64
// or 128).
ctof_status plane_map(CUtensorMap* m, const float2* base, int nplanes, int h, int rows, size_t ld_kx, size_t ld_row,
                      int b0, int b1, int b2) {
  const unsigned long long dims[3] = {(unsigned long long)nplanes, (unsigned long long)h, (unsigned long long)rows};
  const unsigned long long strides[2] = {ld_kx * sizeof(float2), ld_row * sizeof(float2)};
  const unsigned box[3] = {(unsigned)b0, (unsigned)b1, (unsigned)b2};
  return ctof_encode_map(m, 8, 3, base, dims, strides, box, b0 * (int)sizeof(float2));
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

// Row-pass map over inter[row][kx][plane]: boxes of 16 planes x rkx(P) kx x 1 row.
ctof_status row_map(const ctof_kernel_s* k, CUtensorMap* m, const float2* inter, int nplanes, int rows) {
  const size_t LP = plane_ld(nplanes);
  return plane_map(m, inter, nplanes, k->h, rows, LP, (size_t)k->hp * LP, RP, rkx(k->p), 1);
}

}  // namespace

ctof_status ctof_encode_map(CUtensorMap* map, int elem_bytes, int rank, const void* base,
                            const unsigned long long* dims, const unsigned long long* strides_bytes,
                            const unsigned* box, int swizzle_bytes) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) {
    ctof_set_last_error_text("cuTensorMapEncodeTiled is not available from the driver");
    return CTOF_ECUDA;
  }
  if (rank < 1 || rank > 5 || (reinterpret_cast<uintptr_t>(base) & 15)) return CTOF_EINVAL;
  cuuint64_t d[5], s[4];
  cuuint32_t b[5], es[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    es[i] = 1;
    if (i + 1 < rank) {
      if (strides_bytes[i] & 15) return CTOF_EINVAL;
      s[i] = strides_bytes[i];
    }
  }
  const CUtensorMapDataType dt = elem_bytes == 8   ? CU_TENSOR_MAP_DATA_TYPE_UINT64
                                 : elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32
                                 : elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  const CUtensorMapSwizzle sw = swizzle_bytes == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                                : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                : swizzle_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                                      : CU_TENSOR_MAP_SWIZZLE_NONE;
  const CUresult r = enc(map, dt, (cuuint32_t)rank, const_cast<void*>(base), d, s, b, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    ctof_set_last_error_text("cuTensorMapEncodeTiled rejected a tensor map");
    return CTOF_ECUDA;
  }
  return CTOF_OK;
}

ctof_status fft_rows_forward(const ctof_kernel_s* k, const float* in, int nplanes, int rows, int cols_in,
                             int ld_in, float2* inter, cudaStream_t st) {
  if (nplanes <= 0 || rows <= 0) return CTOF_OK;
  CUtensorMap map;
  CTOF_TRY(row_map(k, &map, inter, nplanes, rows));
  const size_t sm = row_smem_bytes(k->p);
  CTOF_P_SWITCH(k->p, {
    CTOF_CUDA_TRY(allow_smem(k_rows_fwd<P_>, sm));
    k_rows_fwd<P_><<<row_grid(rows, nplanes), ROW_WARPS * 32, sm, st>>>(map, in, nplanes, rows, cols_in, ld_in,
                                                                         k->d_tw);
  });
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status fft_rows_inverse(const ctof_kernel_s* k, const float2* inter, int nplanes, int rows, int cols_out,
                             float* out, int ld_out, cudaStream_t st) {
  if (nplanes <= 0 || rows <= 0) return CTOF_OK;
  CUtensorMap map;
  CTOF_TRY(row_map(k, &map, inter, nplanes, rows));
  const size_t sm = row_smem_bytes(k->p);
  const float scale = 1.0f / ((float)k->p * (float)k->p);
  CTOF_P_SWITCH(k->p, {
    CTOF_CUDA_TRY(allow_smem(k_rows_inv<P_, false>, sm));
    k_rows_inv<P_, false><<<row_grid(rows, nplanes), ROW_WARPS * 32, sm, st>>>(
        map, nplanes, rows, cols_out, out, ld_out, scale, k->d_tw, k->d_flags, k->max_polls, nullptr);
  });
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status fft_rows_inverse_norm(const ctof_kernel_s* k, const float2* inter, int nplanes, int rows, int cols_out,
                                  const float* ref, int ld_ref, double* acc, cudaStream_t st) {
  if (nplanes <= 0 || rows <= 0) return CTOF_OK;
  CUtensorMap map;
  CTOF_TRY(row_map(k, &map, inter, nplanes, rows));
  const size_t sm = row_smem_bytes(k->p);
  const float scale = 1.0f / ((float)k->p * (float)k->p);
  CTOF_P_SWITCH(k->p, {
    CTOF_CUDA_TRY(allow_smem(k_rows_inv<P_, true>, sm));
    k_rows_inv<P_, true><<<row_grid(rows, nplanes), ROW_WARPS * 32, sm, st>>>(
        map, nplanes, rows, cols_out, const_cast<float*>(ref), ld_ref, scale, k->d_tw, k->d_flags, k->max_polls,
        acc);
  });
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status fft_rows_admm_t(const ctof_kernel_s* k, float2* inter, const float* m, float* u1, float inv_scale,
                            float rho, cudaStream_t st) {
  CUtensorMap map;
  CTOF_TRY(row_map(k, &map, inter, k->nt, k->n));
  const size_t sm = row_smem_bytes(k->p);
  const float scale = 1.0f / ((float)k->p * (float)k->p);
  CTOF_P_SWITCH(k->p, {
    CTOF_CUDA_TRY(allow_smem(k_rows_admm_t<P_, false>, sm));
    k_rows_admm_t<P_, false><<<row_grid(k->n, k->nt), ROW_WARPS * 32, sm, st>>>(
        map, k->nt, k->n, m, u1, scale, inv_scale, rho, k->d_tw, k->d_flags, k->max_polls);
  });
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status fft_rows_resid_t(const ctof_kernel_s* k, float2* inter, const float* m, cudaStream_t st) {
  CUtensorMap map;
  CTOF_TRY(row_map(k, &map, inter, k->nt, k->n));
  const size_t sm = row_smem_bytes(k->p);
  const float scale = 1.0f / ((float)k->p * (float)k->p);
  CTOF_P_SWITCH(k->p, {
    CTOF_CUDA_TRY(allow_smem(k_rows_admm_t<P_, true>, sm));
    k_rows_admm_t<P_, true><<<row_grid(k->n, k->nt), ROW_WARPS * 32, sm, st>>>(
        map, k->nt, k->n, m, nullptr, scale, 0.f, 0.f, k->d_tw, k->d_flags, k->max_polls);
  });
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

namespace {

// Tile codes: PB for NC = 32 (8, 16), 100 + PB for NC = 16 (108, 116).
#define CTOF_COLS_CASE(KERN, PB_, NC_, ...)                                \
  CTOF_P_SWITCH(k->p, {                                                    \
    CTOF_CUDA_TRY(allow_smem(KERN<P_, PB_, NC_>, sm));                     \
    KERN<P_, PB_, NC_><<<grid, COL_THREADS, sm, st>>>(__VA_ARGS__);        \
  })

#define CTOF_COLS_LAUNCH(KERN, ...)                                                      \
  do {                                                                                   \
    const size_t sm = col_smem_bytes(k->p, nc);                                          \
    dim3 grid(ctof_div_up(k->h, nc / pb), ctof_div_up(nplanes, pb));                     \
    switch (code) {                                                                      \
      case 16: CTOF_COLS_CASE(KERN, 16, 32, __VA_ARGS__); break;                         \
      case 116: CTOF_COLS_CASE(KERN, 16, 16, __VA_ARGS__); break;                        \
      case 108: CTOF_COLS_CASE(KERN, 8, 16, __VA_ARGS__); break;                         \
      default: CTOF_COLS_CASE(KERN, 8, 32, __VA_ARGS__);                                 \
    }                                                                                    \
  } while (0)

// Plane tile (planes per tile, columns per tile) of a tile code.
void tile_of(int& code, int& pb, int& nc) {
  if (code != 16 && code != 108 && code != 116) code = 8;
  pb = code >= 100 ? code - 100 : code;
  nc = code >= 100 ? 16 : 32;
}

}  // namespace

ctof_status fft_cols_forward_pb(const ctof_kernel_s* k, const float2* inter, int nplanes, int rows_in, float2* out,
                                int ldf, int code, cudaStream_t st) {
  if (nplanes <= 0) return CTOF_OK;
  int pb, nc;
  tile_of(code, pb, nc);
  const int P = k->p, rb = P < 256 ? P : 256;
  const size_t LP = plane_ld(nplanes);
  CUtensorMap src, dst;
  CTOF_TRY(plane_map(&src, inter, nplanes, k->h, rows_in, LP, (size_t)k->hp * LP, pb, 1, rb));
  CTOF_TRY(plane_map(&dst, out, nplanes, k->h, P, ldf, (size_t)k->h * ldf, pb, 1, rb));
  CTOF_COLS_LAUNCH(k_cols_fwd, src, dst, rows_in, k->h, k->d_tw, k->d_flags, k->max_polls);
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
  int pb, nc;
  tile_of(code, pb, nc);
  const int P = k->p, rb = P < 256 ? P : 256;
  const size_t LP = plane_ld(nplanes);
  CUtensorMap src, dst;
  CTOF_TRY(plane_map(&src, in, nplanes, k->h, P, ldf, (size_t)k->h * ldf, pb, 1, rb));
  CTOF_TRY(plane_map(&dst, inter, nplanes, k->h, rows_out, LP, (size_t)k->hp * LP, pb, 1, rb));
  CTOF_COLS_LAUNCH(k_cols_inv, src, dst, rows_out, k->h, k->d_tw, k->d_flags, k->max_polls);
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
    } else if (i < tw4_base(p)) {
      const int e = i - p - 31;
      j = ((e & 31) * (e / 32 + 1)) & (p - 1);
    } else if (i < tw_count(p)) {
      const int e = i - tw4_base(p);
      j = ((p / 32) * (e & 7) * (e / 8 + 1)) & (p - 1);
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
