// Learned form: an unrolled proximal-gradient solver whose proximal step is a
// small 3-D CNN, trained on the GPU by this file's own forward and backward
// kernels (no cuDNN/cuBLAS).  Stages s = 0..S-1 from x_0 = 0, or from the
// per-frequency Tikhonov solution T m of the measurement (the library's
// Tikhonov solver, lambda = x0_lambda_rel * max Gram diagonal):
//   g_s     = A_n^T (A_n x_s - m_n)          (the library's forward/adjoint, A_n = A/scale)
//   z_s     = x_s - eta_s g_s
//   x_{s+1} = z_s + mu0 f(z_s / mu0)
// f = conv(1->16)+b, ReLU, conv(16->16)+b, ReLU, conv(16->16)+b, ReLU,
// conv(16->1)+b; 3x3x3 taps, zero padding on each N x N x Z volume; weights
// shared across stages; loss mean(((x_S - mu)/mu0)^2); Adam on FP32 masters.
// Inference may end with data-consistency steps x <- x - T(A x - m).
//
// Activations are BF16, channels-last ([voxel][16]); every layer runs as a
// 16 -> 16 convolution (the single input / output channel of the first and
// last layers padded with zero weights) on warp-level m16n8k16 BF16 MMAs with
// FP32 accumulation: one warp computes 16 voxels along x x 16 output channels,
// K = 27 taps x 16 input channels.  The data gradient is the same kernel with
// flipped taps and transposed channels; the weight gradient is a K = voxels
// MMA reduction with per-CTA partial sums.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <new>
#include <vector>

#include "bulk.cuh"
#include "ctof_internal.h"
#include "umma.cuh"

namespace {

constexpr int CH = 16;
constexpr float MU0 = 0.01f;
constexpr int NLAYER = 4;
const int LAYER_IN[NLAYER] = {1, CH, CH, CH};
const int LAYER_OUT[NLAYER] = {CH, CH, CH, 1};

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned relu2(unsigned v) {
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&v);
  h = __hmax2(h, __floats2bfloat162_rn(0.f, 0.f));
  return *reinterpret_cast<unsigned*>(&h);
}
__device__ __forceinline__ unsigned pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  __nv_bfloat162 h;
  h.x = lo;
  h.y = hi;
  return *reinterpret_cast<unsigned*>(&h);
}

struct Geo {
  int b, z, y, x;  // batch, depth, rows, columns (x % 16 == 0)
};

// Voxel index of (v's row + offsets) or -1 outside the volume.
__device__ __forceinline__ long long neighbour(const Geo& G, int bb, int zz, int yy, int xx) {
  if (zz < 0 || zz >= G.z || yy < 0 || yy >= G.y || xx < 0 || xx >= G.x) return -1;
  return (((long long)bb * G.z + zz) * G.y + yy) * G.x + xx;
}

// One CTA computes an 8-row x TX-voxel patch of one (batch, depth) plane for
// all 16 output channels: the 3 x 10 x (TX+2) input block (halo included,
// zero outside the volume) and the 27 x 16 x 16 weights are staged in shared
// memory with 16-byte cp.async copies; each warp owns one output row and
// runs, per tap, one ldmatrix for the weights and one per 16-voxel job for
// the inputs, then two m16n8k16 MMAs per job.  The two 16-byte halves of a
// voxel's 32-byte channel vector swap places on bit 2 of the voxel index, so
// the eight rows of every ldmatrix land in distinct bank groups.
//   out[v][co] = bias[co] + sum_tap sum_ci W[tap][co][ci] act(in[v + off(tap)][ci])
// act = ReLU if relu_in (applied once to the staged tile); out *= (mask[v][co] > 0) if mask.  IN_F32: the input
// is one FP32 channel `in_f` scaled by in_scale (channel 0; the rest zero).
// OUT_PROX: instead of `out`, x[v] = z[v] + mu0 * bf16(out[v][0]).
constexpr int CV_TY = 8;
constexpr int CV_THREADS = 256;

__device__ __forceinline__ unsigned su32(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void cp16_zfill(void* s, const void* g, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(su32(s)), "l"(g), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void ldm_x4(unsigned (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(su32(p)));
}
// byte offset of 16-byte half h of staged row v
__device__ __forceinline__ int tile_off(int v, int h) { return v * 32 + ((h ^ ((v >> 2) & 1)) << 4); }

size_t conv_smem_bytes(int txc) { return (size_t)3 * (CV_TY + 2) * (16 * txc + 2) * 32 + 27 * CH * 32; }

template <int TXC, bool IN_F32, bool OUT_PROX>
__global__ void __launch_bounds__(CV_THREADS) k_conv3d(const __nv_bfloat16* __restrict__ in,
                                                       const float* __restrict__ in_f, float in_scale, int relu_in,
                                                       const __nv_bfloat16* __restrict__ w,
                                                       const float* __restrict__ bias,
                                                       const __nv_bfloat16* __restrict__ mask,
                                                       __nv_bfloat16* __restrict__ out, const float* __restrict__ z,
                                                       float* __restrict__ x_out, Geo G) {
  constexpr int TX = 16 * TXC, SX = TX + 2, SY = CV_TY + 2;
  extern __shared__ __align__(128) char sm[];
  char* s_in = sm;                      // [3][SY][SX] staged voxels, 32 B each
  char* s_w = sm + 3 * SY * SX * 32;    // [27 * 16] rows (tap, co) of 16 ci, 32 B each
  const int bb = blockIdx.z / G.z, zz = blockIdx.z - bb * G.z;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * CV_TY;
  for (int i = threadIdx.x; i < 27 * CH * 2; i += CV_THREADS)
    cp16_zfill(s_w + tile_off(i >> 1, i & 1), w + (i >> 1) * CH + (i & 1) * 8, true);
  const int nvox = 3 * SY * SX;
  if (IN_F32) {
    for (int v = threadIdx.x; v < nvox; v += CV_THREADS) {
      const int tx = v % SX, r = v / SX, ty = r % SY, tz = r / SY;
      const int gx = x0 + tx - 1, gy = y0 + ty - 1, gz = zz + tz - 1;
      float val = 0.f;
      if (gx >= 0 && gx < G.x && gy >= 0 && gy < G.y && gz >= 0 && gz < G.z)
        val = in_f[(((long long)bb * G.z + gz) * G.y + gy) * G.x + gx] * in_scale;
      *reinterpret_cast<uint4*>(s_in + tile_off(v, 0)) =
          make_uint4(pack2(__float2bfloat16_rn(val), __float2bfloat16_rn(0.f)), 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(s_in + tile_off(v, 1)) = make_uint4(0u, 0u, 0u, 0u);
    }
  } else {
    for (int i = threadIdx.x; i < nvox * 2; i += CV_THREADS) {
      const int v = i >> 1, h = i & 1;
      const int tx = v % SX, r = v / SX, ty = r % SY, tz = r / SY;
      const int gx = x0 + tx - 1, gy = y0 + ty - 1, gz = zz + tz - 1;
      const bool ok = gx >= 0 && gx < G.x && gy >= 0 && gy < G.y && gz >= 0 && gz < G.z;
      const long long gv = ok ? (((long long)bb * G.z + gz) * G.y + gy) * G.x + gx : 0;
      cp16_zfill(s_in + tile_off(v, h), in + gv * CH + h * 8, ok);
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  if (!IN_F32 && relu_in) {  // ReLU once per staged value instead of once per tap
    for (int i = threadIdx.x; i < nvox * 2; i += CV_THREADS) {
      uint4* p = reinterpret_cast<uint4*>(s_in + i * 16);
      uint4 v = *p;
      v.x = relu2(v.x);
      v.y = relu2(v.y);
      v.z = relu2(v.z);
      v.w = relu2(v.w);
      *p = v;
    }
    __syncthreads();
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tg = lane & 3;
  const int mi = lane >> 3, lr = lane & 7;
  const int a_vox = lr + ((mi & 1) << 3), a_half = mi >> 1;   // A: (voxels 0-7 | 8-15) x (ci 0-7 | 8-15)
  const int b_row = lr + ((mi >> 1) << 3), b_half = mi & 1;   // B: (co 0-7 | 8-15) x (ci 0-7 | 8-15)
  float acc[TXC][2][4];
#pragma unroll
  for (int j = 0; j < TXC; ++j)
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[j][n][e] = 0.f;
#pragma unroll 3
  for (int tap = 0; tap < 27; ++tap) {
    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
    unsigned b[4];
    ldm_x4(b, s_w + tile_off(tap * CH + b_row, b_half));
    const int vrow = (dz * SY + warp + dy) * SX + dx;
    // +16 voxels keeps bit 2 of the voxel index, so job j is 512 bytes further on
    const char* a_base = s_in + tile_off(vrow + a_vox, a_half);
#pragma unroll
    for (int j = 0; j < TXC; ++j) {
      unsigned a[4];
      ldm_x4(a, a_base + j * 512);
      mma_bf16(acc[j][0], a, b[0], b[1]);
      if (!OUT_PROX) mma_bf16(acc[j][1], a, b[2], b[3]);  // the last layer has one output channel
    }
  }
  const int yy = y0 + warp;
  const long long row = (((long long)bb * G.z + zz) * G.y + yy) * G.x;
#pragma unroll
  for (int j = 0; j < TXC; ++j) {
    const long long v0 = row + x0 + j * 16 + g, v1 = v0 + 8;
    if (OUT_PROX) {
      if (tg == 0) {
        const float b0 = bias ? bias[0] : 0.f;
        const float f0 = __bfloat162float(__float2bfloat16_rn(acc[j][0][0] + b0));
        const float f1 = __bfloat162float(__float2bfloat16_rn(acc[j][0][2] + b0));
        x_out[v0] = z[v0] + MU0 * f0;
        x_out[v1] = z[v1] + MU0 * f1;
      }
      continue;
    }
    unsigned* outw = reinterpret_cast<unsigned*>(out);
    const unsigned* maskw = reinterpret_cast<const unsigned*>(mask);
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int co = nt * 8 + 2 * tg;
      float r0 = acc[j][nt][0], r1 = acc[j][nt][1], r2 = acc[j][nt][2], r3 = acc[j][nt][3];
      if (bias) {
        r0 += bias[co];
        r1 += bias[co + 1];
        r2 += bias[co];
        r3 += bias[co + 1];
      }
      if (mask) {
        const unsigned m0 = maskw[v0 * 8 + (co >> 1)], m1 = maskw[v1 * 8 + (co >> 1)];
        const float2 f0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&m0));
        const float2 f1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&m1));
        r0 = f0.x > 0.f ? r0 : 0.f;
        r1 = f0.y > 0.f ? r1 : 0.f;
        r2 = f1.x > 0.f ? r2 : 0.f;
        r3 = f1.y > 0.f ? r3 : 0.f;
      }
      outw[v0 * 8 + (co >> 1)] = pack2(__float2bfloat16_rn(r0), __float2bfloat16_rn(r1));
      outw[v1 * 8 + (co >> 1)] = pack2(__float2bfloat16_rn(r2), __float2bfloat16_rn(r3));
    }
  }
}

// ---- hidden layers at inference on tcgen05 ----
//
// out[v][co] = act(bias[co] + sum_tap sum_ci W[tap][co][ci] in[v + off(tap)][ci])
// on the tensor cores, M = 128 voxels along x, K = 16 input channels (the
// input is stored after its ReLU).  A work unit is TCV_YB output rows of one
// (volume, depth, x segment); warp 0 (one thread) streams the unit's input rows
// (y0 - 1 .. y0 + TCV_YB, each as its three depth planes of 130 voxels x0 - 1 ..
// x0 + 128, one tensor-map box of 32-byte voxel rows per plane in the copy
// engine's 32-byte swizzle) into a ring of TCV_RING slots (zero fill outside
// the volume).  Warp 1 (one thread) issues the MMAs input row by input row:
// each of the row's nine (depth, x shift) A views (the plane's voxel rows as a
// K-major operand in the same swizzle, the x shift a 32-byte start offset) is
// multiplied by the weights of
// its three dy taps stacked along N, so one MMA (N = 48) feeds output rows
// j - 2, j - 1, j of input row j, held in three consecutive accumulators of a
// TCV_NACC-slot TMEM ring (split into two MMAs where they wrap around the
// ring).  An M = 128, K = 16 MMA costs the same issue time for every N up to
// about 90, so nine N = 48 MMAs per input row replace the 27 N = 16 MMAs per
// output row of a tap-by-tap loop.  Every MMA accumulates: warps 4-7 drain an
// accumulator (bias, ReLU or the fused residual step x = z + mu0 bf16(out[v][0]),
// store) and zero it, and zero all slots at the start.  mbarrier hand-offs with
// bounded waits; 96 TMEM columns, three CTAs per SM.
constexpr int TCV_RING = 4;
constexpr int TCV_YB = 32;
constexpr int TCV_NACC = 6;                     // accumulator ring slots (16 columns each)
constexpr int TCV_PL = 17 * 256;                // bytes of one staged plane (130 voxel rows of 32 bytes, padded)
constexpr int TCV_SLOT = 3 * TCV_PL;            // one staged input row: 3 depth planes
constexpr int TCV_BT = 48 * 32;                 // bytes of one stacked weight tile (48 rows x 16 ci)
constexpr int TCV_WB = 9 * TCV_BT;
constexpr int TCV_THREADS = 256;
constexpr int TCV_LOAD = 3 * 130 * 32;          // bytes landing per staged row
constexpr size_t TCV_SMEM = 1024 + TCV_RING * TCV_SLOT + TCV_WB + 64 + 256;

__host__ __device__ constexpr uint32_t tcv_idesc(int n) {  // kind::f16: D F32, A / B BF16, M = 128
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// D += A x B, both from shared memory; always accumulating.
__device__ __forceinline__ void tcv_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(1u)
      : "memory");
}

__device__ __forceinline__ bool tcv_wait(uint64_t* bar, uint32_t parity, long long max_polls, volatile int* abort_w,
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

// Warp-level bounded wait: lane 0 polls, the others acquire with one poll.
__device__ __forceinline__ bool tcv_wait_warp(uint64_t* bar, uint32_t parity, long long max_polls,
                                              volatile int* abort_w, int* flag, int lane) {
  int ok = 1;
  if (lane == 0) ok = tcv_wait(bar, parity, max_polls, abort_w, flag) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok && lane != 0) (void)bulk::try_wait(bar, parity);
  return ok != 0;
}

__device__ __forceinline__ void tcv_zero16(uint32_t taddr) {
  const uint32_t zero[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  umma::tmem_st8(taddr, zero);
  umma::tmem_st8(taddr + 8, zero);
}

template <bool PROX>
__global__ void __launch_bounds__(TCV_THREADS, 1)
    k_conv3d_tc(const __grid_constant__ CUtensorMap amap, const __nv_bfloat16* __restrict__ w,
                const float* __restrict__ bias, __nv_bfloat16* __restrict__ out, const float* __restrict__ z,
                float* __restrict__ x_out, Geo G, int* flag, long long max_polls) {
  extern __shared__ float4 tcv_smem4[];
  unsigned char* sm;
  {
    const uint32_t s = bulk::saddr(tcv_smem4);
    sm = reinterpret_cast<unsigned char*>(tcv_smem4) + (((s + 1023u) & ~1023u) - s);
  }
  unsigned char* ring = sm;
  unsigned char* s_w = sm + TCV_RING * TCV_SLOT;
  float* s_bias = reinterpret_cast<float*>(s_w + TCV_WB);
  uint64_t* bar = reinterpret_cast<uint64_t*>(s_bias + 16);
  uint64_t* slot_full = bar;                   // [RING], one arrival + the copies' bytes
  uint64_t* slot_empty = bar + TCV_RING;       // [RING], the MMAs that read the row (commit)
  uint64_t* acc_full = bar + 2 * TCV_RING;     // [NACC], the row's last MMAs (commit)
  uint64_t* acc_empty = acc_full + TCV_NACC;   // [NACC], one arrival per epilogue warp (slot zeroed)
  uint64_t* drain_bar = acc_empty + TCV_NACC;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain_bar + 1);
  volatile int* abort_w = reinterpret_cast<volatile int*>(drain_bar + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // stacked weights, K-major B operand of 48 rows in the 32-byte swizzle: tile
  // (dz, dx) holds rows n = 16 blk + co with dy = 2 - blk, row n at n 32 bytes,
  // its 16-byte half g (input channels 8 g ..) at half g ^ ((n / 4) & 1)
  for (int i = threadIdx.x; i < 27 * 16 * 2; i += TCV_THREADS) {
    const int t = i >> 5, co = (i >> 1) & 15, g = i & 1;
    const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3, n = (2 - dy) * 16 + co;
    *reinterpret_cast<uint4*>(s_w + (dz * 3 + dx) * TCV_BT + n * 32 + ((g ^ ((n >> 2) & 1)) << 4)) =
        *reinterpret_cast<const uint4*>(w + ((size_t)t * CH + co) * CH + 8 * g);
  }
  if (threadIdx.x < 16) s_bias[threadIdx.x] = bias ? bias[threadIdx.x] : 0.f;
  if (threadIdx.x == 0) {
    for (int i = 0; i < TCV_RING; ++i) {
      bulk::bar_init(slot_full + i, 1);
      bulk::bar_init(slot_empty + i, 1);
    }
    for (int i = 0; i < TCV_NACC; ++i) {
      bulk::bar_init(acc_full + i, 1);
      bulk::bar_init(acc_empty + i, 4);
    }
    bulk::bar_init(drain_bar, 1);
    *abort_w = 0;
  }
  if (warp == 0) umma::tmem_alloc(tslot, 128);
  umma::fence_proxy_async();  // the weights, before the MMAs read them
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t taddr = *tslot;
  const int nseg = (G.x + 127) / 128, nyb = (G.y + TCV_YB - 1) / TCV_YB;
  const int nunits = G.b * G.z * nyb * nseg;
  auto unit_at = [&](int u, int& bb, int& zz, int& y0, int& x0) {
    x0 = (u % nseg) * 128;
    int r = u / nseg;
    y0 = (r % nyb) * TCV_YB;
    r /= nyb;
    zz = r % G.z;
    bb = r / G.z;
  };

  if (warp == 0) {
    // ---------------- producer: input rows y0 - 1 .. y0 + TCV_YB of each unit ----------------
    if (lane == 0) {
      int gr = 0;  // rows staged
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        int bb, zz, y0, x0;
        unit_at(u, bb, zz, y0, x0);
        for (int j = 0; j < TCV_YB + 2; ++j, ++gr) {
          const int s = gr % TCV_RING;
          if (gr >= TCV_RING &&
              !tcv_wait(slot_empty + s, (uint32_t)((gr / TCV_RING) + 1) & 1u, max_polls, abort_w, flag)) {
            ok = false;
            break;
          }
          unsigned char* dst = ring + s * TCV_SLOT;
          bulk::arrive_expect(slot_full + s, TCV_LOAD);
          for (int dz = 0; dz < 3; ++dz)
            bulk::tensor_g2s_5d(dst + dz * TCV_PL, &amap, 0, x0 - 1, y0 - 1 + j, zz - 1 + dz, bb, slot_full + s);
        }
      }
      // no copy may still be landing when the CTA ends: the last load into each slot
      for (int s = 0; s < TCV_RING && s < gr; ++s)
        bulk::wait(slot_full + s, (uint32_t)((gr - 1 - s) / TCV_RING) & 1u, bulk::DRAIN_POLLS);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      // slot 0, plane 0, x shift 0: 32-byte voxel rows, 8-row groups 256 bytes apart, 32-byte swizzle
      const uint64_t a_desc0 = umma::desc(bulk::saddr(ring), 16, 256) | (6ull << 61);
      // tile (0, 0) from output row j - 2; 8-row groups 256 bytes apart, 32-byte swizzle (layout 6)
      const uint64_t b_desc0 = umma::desc(bulk::saddr(s_w), 16, 256) | (6ull << 61);
      int gr = 0, gbase = 0;  // input rows consumed, first output row of the unit
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x, gbase += TCV_YB) {
        for (int j = 0; j < TCV_YB + 2 && ok; ++j, ++gr) {
          const int s = gr % TCV_RING;
          if (j < TCV_YB) {  // output row j enters: its accumulator is drained and zeroed
            const int gi = gbase + j;
            if (!tcv_wait(acc_empty + gi % TCV_NACC, (uint32_t)(gi / TCV_NACC) & 1u, max_polls, abort_w, flag)) {
              ok = false;
              break;
            }
          }
          if (!tcv_wait(slot_full + s, (uint32_t)(gr / TCV_RING) & 1u, max_polls, abort_w, flag)) {
            ok = false;
            break;
          }
          umma::fence_after_sync();
          const int lo = j - 2 > 0 ? j - 2 : 0, hi = j < TCV_YB - 1 ? j : TCV_YB - 1;
          const int cnt = hi - lo + 1, s0 = (gbase + lo) % TCV_NACC;
          const int first = cnt < TCV_NACC - s0 ? cnt : TCV_NACC - s0;
          const uint32_t d0 = taddr + 16 * s0, id0 = tcv_idesc(16 * first);
          const uint32_t id1 = tcv_idesc(16 * (cnt - first > 0 ? cnt - first : 1));
          const uint64_t boff0 = (uint64_t)((512 * (lo - j + 2)) >> 4);  // 16 rows = 512 bytes
          const uint64_t boff1 = (uint64_t)((512 * (lo + first - j + 2)) >> 4);
          const uint64_t arow = a_desc0 + (uint64_t)((s * TCV_SLOT) >> 4);
#pragma unroll
          for (int dz = 0; dz < 3; ++dz)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
              const uint64_t av = arow + (uint64_t)((dz * TCV_PL + dx * 32) >> 4);
              const uint64_t bt = b_desc0 + (uint64_t)(((dz * 3 + dx) * TCV_BT) >> 4);
              tcv_mma(d0, av, bt + boff0, id0);
              if (first < cnt) tcv_mma(taddr, av, bt + boff1, id1);
            }
          umma::commit(slot_empty + s);                                    // the staged row is read
          if (j >= 2) umma::commit(acc_full + (gbase + j - 2) % TCV_NACC);  // output row j - 2 is complete
        }
      }
      umma::commit(drain_bar);
      bulk::wait(drain_bar, 0, bulk::DRAIN_POLLS);
    }
  } else if (warp >= 4) {
    // ---------------- epilogue: bias, activation, store; zero the accumulator ----------------
    const int r = 32 * (warp & 3) + lane;  // TMEM lane = voxel of the 128-row
    const uint32_t trow = taddr + ((uint32_t)(32 * (warp & 3)) << 16);
    for (int a = 0; a < TCV_NACC; ++a) tcv_zero16(trow + 16 * a);
    umma::tmem_wait_st();
    umma::fence_before_sync();
    __syncwarp();
    if (lane == 0)
      for (int a = 0; a < TCV_NACC; ++a) bulk::arrive(acc_empty + a);
    int go = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      int bb, zz, y0, x0;
      unit_at(u, bb, zz, y0, x0);
      for (int j = 0; j < TCV_YB; ++j, ++go) {
        const int a = go % TCV_NACC;
        if (!tcv_wait_warp(acc_full + a, (uint32_t)(go / TCV_NACC) & 1u, max_polls, abort_w, flag, lane)) {
          ok = false;
          break;
        }
        umma::fence_after_sync();
        float d[16];
        umma::tmem_ld16(trow + 16 * a, d);
        tcv_zero16(trow + 16 * a);
        umma::tmem_wait_st();
        umma::fence_before_sync();
        __syncwarp();
        if (lane == 0) bulk::arrive(acc_empty + a);
        const int yy = y0 + j, xx = x0 + r;
        if (yy < G.y && xx < G.x) {
          const long long v = (((long long)bb * G.z + zz) * G.y + yy) * G.x + xx;
          if (PROX) {
            const float f0 = __bfloat162float(__float2bfloat16_rn(d[0] + s_bias[0]));
            x_out[v] = z[v] + MU0 * f0;
          } else {
            unsigned p[8];
#pragma unroll
            for (int e = 0; e < 8; ++e)
              p[e] = pack2(__float2bfloat16_rn(fmaxf(d[2 * e] + s_bias[2 * e], 0.f)),
                           __float2bfloat16_rn(fmaxf(d[2 * e + 1] + s_bias[2 * e + 1], 0.f)));
            uint4* o = reinterpret_cast<uint4*>(out + v * CH);
            o[0] = make_uint4(p[0], p[1], p[2], p[3]);
            o[1] = make_uint4(p[4], p[5], p[6], p[7]);
          }
        }
      }
    }
  }
  __syncwarp();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (warp == 0) umma::tmem_dealloc(taddr, 128);
}

// First layer at inference: one input channel (z / mu0), so the 27 taps (padded
// to 32) form the MMA's K dimension instead of 27 K = 16 channel blocks with
// 15 zero channels: 2 x 2 MMAs per 16-voxel job instead of 27 x 2.  The input
// tile holds one BF16 value per voxel; A fragments are gathered from it tap by
// tap, B fragments (W1[co][tap]) sit in registers for the whole CTA.
template <int TXC, bool RELU_OUT>
__global__ void __launch_bounds__(CV_THREADS) k_conv_first(const float* __restrict__ zin, float in_scale,
                                                           const __nv_bfloat16* __restrict__ w,
                                                           const float* __restrict__ bias,
                                                           __nv_bfloat16* __restrict__ out, Geo G) {
  constexpr int TX = 16 * TXC, SX = TX + 2, SY = CV_TY + 2;
  __shared__ __nv_bfloat16 s_in[3 * SY * SX];
  const int bb = blockIdx.z / G.z, zz = blockIdx.z - bb * G.z;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * CV_TY;
  for (int v = threadIdx.x; v < 3 * SY * SX; v += CV_THREADS) {
    const int tx = v % SX, r = v / SX, ty = r % SY, tz = r / SY;
    const int gx = x0 + tx - 1, gy = y0 + ty - 1, gz = zz + tz - 1;
    float val = 0.f;
    if (gx >= 0 && gx < G.x && gy >= 0 && gy < G.y && gz >= 0 && gz < G.z)
      val = zin[(((long long)bb * G.z + gz) * G.y + gy) * G.x + gx] * in_scale;
    s_in[v] = __float2bfloat16_rn(val);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tg = lane & 3;
  const __nv_bfloat16 zb = __float2bfloat16_rn(0.f);
  // B[k = tap][n = co] = W1[co][tap] (tap >= 27: 0); [k chunk][n tile][b0 / b1]
  unsigned bf[2][2][2];
  // this lane's taps: k chunk kc, half h, element e -> tap 16 kc + 8 h + 2 tg + e; offset in the tile or -1
  int toff[2][2][2];
#pragma unroll
  for (int kc = 0; kc < 2; ++kc)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int t = 16 * kc + 8 * h + 2 * tg + e;
        toff[kc][h][e] = t < 27 ? ((t / 9) * SY + (t / 3) % 3) * SX + t % 3 : -1;
      }
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int co = nt * 8 + g, t = 16 * kc + 8 * h + 2 * tg;
        const __nv_bfloat16 lo = t < 27 ? w[(t * CH + co) * CH] : zb;
        const __nv_bfloat16 hi = t + 1 < 27 ? w[((t + 1) * CH + co) * CH] : zb;
        bf[kc][nt][h] = pack2(lo, hi);
      }
    }
  __syncthreads();
  float acc[TXC][2][4];
#pragma unroll
  for (int j = 0; j < TXC; ++j)
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[j][n][e] = 0.f;
#pragma unroll
  for (int j = 0; j < TXC; ++j) {
    const int base0 = warp * SX + j * 16 + g, base1 = base0 + 8;
#pragma unroll
    for (int kc = 0; kc < 2; ++kc) {
      unsigned a[4];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int o0 = toff[kc][h][0], o1 = toff[kc][h][1];
        a[2 * h] = pack2(o0 >= 0 ? s_in[base0 + o0] : zb, o1 >= 0 ? s_in[base0 + o1] : zb);
        a[2 * h + 1] = pack2(o0 >= 0 ? s_in[base1 + o0] : zb, o1 >= 0 ? s_in[base1 + o1] : zb);
      }
      mma_bf16(acc[j][0], a, bf[kc][0][0], bf[kc][0][1]);
      mma_bf16(acc[j][1], a, bf[kc][1][0], bf[kc][1][1]);
    }
  }
  const long long row = (((long long)bb * G.z + zz) * G.y + y0 + warp) * G.x;
  unsigned* outw = reinterpret_cast<unsigned*>(out);
#pragma unroll
  for (int j = 0; j < TXC; ++j) {
    const long long v0 = row + x0 + j * 16 + g, v1 = v0 + 8;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int co = nt * 8 + 2 * tg;
      float r0 = acc[j][nt][0] + bias[co], r1 = acc[j][nt][1] + bias[co + 1];
      float r2 = acc[j][nt][2] + bias[co], r3 = acc[j][nt][3] + bias[co + 1];
      if (RELU_OUT) {
        r0 = fmaxf(r0, 0.f);
        r1 = fmaxf(r1, 0.f);
        r2 = fmaxf(r2, 0.f);
        r3 = fmaxf(r3, 0.f);
      }
      outw[v0 * 8 + (co >> 1)] = pack2(__float2bfloat16_rn(r0), __float2bfloat16_rn(r1));
      outw[v1 * 8 + (co >> 1)] = pack2(__float2bfloat16_rn(r2), __float2bfloat16_rn(r3));
    }
  }
}

// Per-CTA partial weight gradients: part[blk][tap][co][ci] = sum over this CTA's
// voxels of dy[v][co] act(x[v + off(tap)][ci]).  Warp w owns taps w, w+8, w+16, w+24.
constexpr int WG_ROWS = 16;  // (b, z, y) rows per CTA
__global__ void __launch_bounds__(256) k_wgrad(const __nv_bfloat16* __restrict__ dy, const __nv_bfloat16* __restrict__ x,
                                               int relu_in, Geo G, float* __restrict__ part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tg = lane & 3;
  const long long rows = (long long)G.b * G.z * G.y;
  const long long r0 = (long long)blockIdx.x * WG_ROWS;
  float acc[4][2][4] = {};
  const __nv_bfloat16* dyb = dy;
  for (long long row = r0; row < r0 + WG_ROWS && row < rows; ++row) {
    const int yy = (int)(row % G.y);
    const int zz = (int)((row / G.y) % G.z);
    const int bb = (int)(row / ((long long)G.y * G.z));
    for (int x0 = 0; x0 < G.x; x0 += 16) {
      const long long vb = neighbour(G, bb, zz, yy, x0);
      // A = dy^T: rows co, cols the 16 voxels
      unsigned a[4];
      a[0] = pack2(dyb[(vb + 2 * tg) * CH + g], dyb[(vb + 2 * tg + 1) * CH + g]);
      a[1] = pack2(dyb[(vb + 2 * tg) * CH + g + 8], dyb[(vb + 2 * tg + 1) * CH + g + 8]);
      a[2] = pack2(dyb[(vb + 2 * tg + 8) * CH + g], dyb[(vb + 2 * tg + 9) * CH + g]);
      a[3] = pack2(dyb[(vb + 2 * tg + 8) * CH + g + 8], dyb[(vb + 2 * tg + 9) * CH + g + 8]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int tap = warp + 8 * j;
        if (tap >= 27) break;
        const int dz = tap / 9 - 1, dy_ = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        const long long n0 = neighbour(G, bb, zz + dz, yy + dy_, x0 + 2 * tg + dx);
        const long long n1 = neighbour(G, bb, zz + dz, yy + dy_, x0 + 2 * tg + 1 + dx);
        const long long n8 = neighbour(G, bb, zz + dz, yy + dy_, x0 + 2 * tg + 8 + dx);
        const long long n9 = neighbour(G, bb, zz + dz, yy + dy_, x0 + 2 * tg + 9 + dx);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int ci = nt * 8 + g;
          const __nv_bfloat16 zb = __float2bfloat16_rn(0.f);
          __nv_bfloat16 e0 = n0 >= 0 ? x[n0 * CH + ci] : zb, e1 = n1 >= 0 ? x[n1 * CH + ci] : zb;
          __nv_bfloat16 e8 = n8 >= 0 ? x[n8 * CH + ci] : zb, e9 = n9 >= 0 ? x[n9 * CH + ci] : zb;
          unsigned b0 = pack2(e0, e1), b1 = pack2(e8, e9);
          if (relu_in) {
            b0 = relu2(b0);
            b1 = relu2(b1);
          }
          mma_bf16(acc[j][nt], a, b0, b1);
        }
      }
    }
  }
  float* p = part + (size_t)blockIdx.x * 27 * CH * CH;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int tap = warp + 8 * j;
    if (tap >= 27) break;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int ci = nt * 8 + 2 * tg;
      p[(tap * CH + g) * CH + ci] = acc[j][nt][0];
      p[(tap * CH + g) * CH + ci + 1] = acc[j][nt][1];
      p[(tap * CH + g + 8) * CH + ci] = acc[j][nt][2];
      p[(tap * CH + g + 8) * CH + ci + 1] = acc[j][nt][3];
    }
  }
}

// acc[i] += sum over blocks of part[blk][i]  (i < 27*16*16)
__global__ void k_reduce_parts(const float* __restrict__ part, int nblk, float* __restrict__ acc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 27 * CH * CH) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += part[(size_t)b * 27 * CH * CH + i];
  acc[i] += s;
}

// db[c] += sum_v dy[v][c]
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ dy, long long nvox, float* __restrict__ db) {
  __shared__ float red[256][CH + 1];
  float s[CH] = {};
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < CH; ++c) s[c] += __bfloat162float(dy[v * CH + c]);
#pragma unroll
  for (int c = 0; c < CH; ++c) red[threadIdx.x][c] = s[c];
  __syncthreads();
  if (threadIdx.x < CH) {
    float t = 0.f;
    for (int i = 0; i < blockDim.x; ++i) t += red[i][threadIdx.x];
    atomicAdd(&db[threadIdx.x], t);
  }
}

// bf16 [v][16] <- (scale * src[v], 0, ..., 0)
__global__ void k_pack1(const float* __restrict__ src, float scale, long long nvox, __nv_bfloat16* __restrict__ out) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
    uint4* o = reinterpret_cast<uint4*>(out + v * CH);
    const unsigned first = pack2(__float2bfloat16_rn(src[v] * scale), __float2bfloat16_rn(0.f));
    o[0] = make_uint4(first, 0u, 0u, 0u);
    o[1] = make_uint4(0u, 0u, 0u, 0u);
  }
}

// z = x - eta[s] * inv_s2 * g_raw, and g = inv_s2 * g_raw stored for the step-size gradient
__global__ void k_zstep(const float* __restrict__ x, float* __restrict__ g, const float* __restrict__ eta, int s,
                        float inv_s2, long long n, float* __restrict__ z) {
  const float e = eta[s];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gv = g[i] * inv_s2;
    g[i] = gv;
    z[i] = x[i] - e * gv;
  }
}

__global__ void k_sub(float* __restrict__ a, const float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a[i] -= b[i];
}

// a -= b over n4 float4 (both 16-byte aligned)
__global__ void k_sub4(float4* __restrict__ a, const float4* __restrict__ b, long long n4) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
    float4 x = a[i];
    const float4 y = b[i];
    x.x -= y.x;
    x.y -= y.y;
    x.z -= y.z;
    x.w -= y.w;
    a[i] = x;
  }
}

// res[b] = sqrt(acc[2b] / acc[2b + 1]); a zero reference gives 0 for a zero
// residual and +inf otherwise.
__global__ void k_ratio_sqrt(const double* __restrict__ acc, int n, double* __restrict__ res) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const double r2 = acc[2 * b], m2 = acc[2 * b + 1];
  res[b] = m2 > 0.0 ? sqrt(r2 / m2) : (r2 > 0.0 ? (double)INFINITY : 0.0);
}

// r = (x - mu)/mu0; loss partial sums; gx = 2 r / (mu0 * ntot)
__global__ void k_loss(const float* __restrict__ x, const float* __restrict__ mu, long long n, float* __restrict__ gx,
                       double* __restrict__ loss_sum) {
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float r = (x[i] - mu[i]) / MU0;
    s += (double)r * r;
    gx[i] = 2.f * r / (MU0 * (float)n);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss_sum, s);
}

// gz = gx + du[v][0] / mu0 ; deta[s] -= sum gz * g
__global__ void k_gz(const float* __restrict__ gx, const __nv_bfloat16* __restrict__ du, const float* __restrict__ g,
                     long long n, float* __restrict__ gz, float* __restrict__ deta, int s) {
  float acc = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float v = gx[i] + __bfloat162float(du[i * CH]) / MU0;
    gz[i] = v;
    acc += v * g[i];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&deta[s], -acc);
}

// gx = gz - eta[s] * inv_s2 * h
__global__ void k_gx(const float* __restrict__ gz, const float* __restrict__ h, const float* __restrict__ eta, int s,
                     float inv_s2, long long n, float* __restrict__ gx) {
  const float e = eta[s];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    gx[i] = gz[i] - e * inv_s2 * h[i];
}

struct LayerOff {
  int w, b, ci, co;
};


// Master FP32 parameters -> padded BF16 forward weights [tap][co][ci], data-gradient
// weights [tap][ci][co] with flipped taps, and padded FP32 biases.
__global__ void k_prep_weights(const float* __restrict__ theta, LayerOff L, __nv_bfloat16* __restrict__ wf,
                               __nv_bfloat16* __restrict__ wb, float* __restrict__ bias) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < CH) bias[i] = i < L.co ? theta[L.b + i] : 0.f;
  if (i >= 27 * CH * CH) return;
  const int tap = i / (CH * CH), co = (i / CH) % CH, ci = i % CH;
  const float v = (co < L.co && ci < L.ci) ? theta[L.w + (co * L.ci + ci) * 27 + tap] : 0.f;
  wf[(tap * CH + co) * CH + ci] = __float2bfloat16_rn(v);
  wb[((26 - tap) * CH + ci) * CH + co] = __float2bfloat16_rn(v);
}

// flat gradient += padded layer gradients
__global__ void k_grad_to_flat(const float* __restrict__ dw, const float* __restrict__ db, LayerOff L,
                               float* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L.co) grad[L.b + i] += db[i];
  if (i >= L.co * L.ci * 27) return;
  const int co = i / (L.ci * 27), ci = (i / 27) % L.ci, tap = i % 27;
  grad[L.w + i] += dw[(tap * CH + co) * CH + ci];
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = gr[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

int grid_for(long long n);

// a -= b (n floats); float4 when both pointers are 16-byte aligned and n % 4 == 0
cudaError_t sub_inplace(float* a, const float* b, long long n, cudaStream_t st) {
  if (((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0 && (n & 3) == 0)
    k_sub4<<<grid_for(n / 4), 256, 0, st>>>(reinterpret_cast<float4*>(a), reinterpret_cast<const float4*>(b), n / 4);
  else
    k_sub<<<grid_for(n), 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

struct ctof_learned_s {
  int stages;
  int nparam;
  ctof_learned_options opt;
  int device;
  LayerOff lo[NLAYER];
  float* d_theta;   // [nparam] FP32 masters
  float* d_grad;
  float* d_m1;
  float* d_m2;
  long long adam_step;
  __nv_bfloat16* d_wf;  // [4][27][16][16]
  __nv_bfloat16* d_wb;
  float* d_bias;        // [4][16]
  float* d_dw;          // [4][27][16][16] FP32 accumulators
  float* d_db;          // [4][16]
  double* d_loss;
  // per-geometry workspace
  void* d_ws;
  size_t ws_bytes;
  long long ws_nvox;
  int ws_batch, ws_nt;
};

namespace {

ctof_status learned_prep(ctof_learned_s* L, cudaStream_t st) {
  for (int l = 0; l < NLAYER; ++l) {
    k_prep_weights<<<(27 * CH * CH + 255) / 256, 256, 0, st>>>(L->d_theta, L->lo[l], L->d_wf + l * 27 * CH * CH,
                                                               L->d_wb + l * 27 * CH * CH, L->d_bias + l * CH);
    CTOF_CUDA_TRY(cudaGetLastError());
  }
  return CTOF_OK;
}

struct Ws {
  float *x, *gx, *gz, *h;
  double* acc;                  // [batch][2] data-residual sums
  float *z, *g;                 // [S][V]
  __nv_bfloat16 *u, *y1, *y2, *y3;  // [S][V][16]
  __nv_bfloat16 *da, *db_;  // [V][16]
  float* part;
  int nblk;
  float2 *spec_t, *spec_z;  // [batch][nf][ldt], [batch][nf][ldz] (or [nf][ldzb], see zb)
  // Z side as one plane-batched FFT over batch * nz planes (batch >= 4, nz even):
  // spectra interleaved per frequency, row pitch ldzb, own FFT intermediate
  float2* inter_zb;
  int ldzb;
};

ctof_status learned_workspace(ctof_learned_s* L, const ctof_kernel_s* k, int batch, bool train, Ws* w) {
  const long long V = (long long)batch * k->nz * k->n * k->n;
  const int S = train ? L->stages : 1;
  const long long rows = (long long)batch * k->nz * k->n;
  const int nblk = (int)((rows + WG_ROWS - 1) / WG_ROWS);
  size_t need = 0;
  auto add = [&](size_t b) {
    const size_t at = need;
    need += (b + 255) & ~(size_t)255;
    return at;
  };
  const size_t o_x = add(V * 4), o_acc = add((size_t)batch * 2 * 8), o_gx = add(V * 4), o_gz = add(V * 4), o_h = add(V * 4);
  const size_t o_z = add((size_t)S * V * 4), o_g = add((size_t)S * V * 4);
  const size_t o_u = add((size_t)S * V * CH * 2), o_y1 = add((size_t)S * V * CH * 2), o_y2 = add((size_t)S * V * CH * 2),
               o_y3 = add((size_t)S * V * CH * 2);
  const size_t o_da = add(V * CH * 2), o_db = add(V * CH * 2);
  const size_t o_p = add((size_t)nblk * 27 * CH * CH * 4);
  const size_t o_st = add((size_t)batch * k->nf * k->ldt * 8), o_sz = add((size_t)batch * k->nf * k->ldz * 8);
  const bool zb = batch >= 4 && (k->nz % 2) == 0;
  const size_t o_izb = add(zb ? fft_inter_elems(k, batch * k->nz, k->n) * 8 : 0);
  if (need > L->ws_bytes) {
    if (L->d_ws) cudaFree(L->d_ws);
    L->d_ws = nullptr;
    L->ws_bytes = 0;
    if (cudaMalloc(&L->d_ws, need) != cudaSuccess) {
      cudaGetLastError();
      return CTOF_ENOMEM;
    }
    L->ws_bytes = need;
  }
  char* b = static_cast<char*>(L->d_ws);
  w->x = reinterpret_cast<float*>(b + o_x);
  w->acc = reinterpret_cast<double*>(b + o_acc);
  w->gx = reinterpret_cast<float*>(b + o_gx);
  w->gz = reinterpret_cast<float*>(b + o_gz);
  w->h = reinterpret_cast<float*>(b + o_h);
  w->z = reinterpret_cast<float*>(b + o_z);
  w->g = reinterpret_cast<float*>(b + o_g);
  w->u = reinterpret_cast<__nv_bfloat16*>(b + o_u);
  w->y1 = reinterpret_cast<__nv_bfloat16*>(b + o_y1);
  w->y2 = reinterpret_cast<__nv_bfloat16*>(b + o_y2);
  w->y3 = reinterpret_cast<__nv_bfloat16*>(b + o_y3);
  w->da = reinterpret_cast<__nv_bfloat16*>(b + o_da);
  w->db_ = reinterpret_cast<__nv_bfloat16*>(b + o_db);
  w->part = reinterpret_cast<float*>(b + o_p);
  w->spec_t = reinterpret_cast<float2*>(b + o_st);
  w->spec_z = reinterpret_cast<float2*>(b + o_sz);
  w->inter_zb = zb ? reinterpret_cast<float2*>(b + o_izb) : nullptr;
  w->ldzb = zb ? ctof_round_up(batch * k->nz, 8) : 0;
  w->nblk = nblk;
  return CTOF_OK;
}

template <bool IN_F32, bool OUT_PROX>
ctof_status conv_launch(const __nv_bfloat16* in, const float* in_f, float in_scale, int relu_in,
                        const __nv_bfloat16* wt, const float* bias, const __nv_bfloat16* mask, __nv_bfloat16* out,
                        const float* z, float* x_out, Geo G, cudaStream_t st) {
  // 32-voxel-wide tiles (47 KB of shared memory) let four CTAs share an SM
  const int txc = G.x % 32 == 0 ? 2 : 1;
  const dim3 grid(G.x / (16 * txc), G.y / CV_TY, G.b * G.z);
  const size_t smem = conv_smem_bytes(txc);
  switch (txc) {
#define CTOF_CONV_CASE(T)                                                                                       \
  case T:                                                                                                       \
    CTOF_CUDA_TRY(cudaFuncSetAttribute(k_conv3d<T, IN_F32, OUT_PROX>,                                          \
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));               \
    k_conv3d<T, IN_F32, OUT_PROX><<<grid, CV_THREADS, smem, st>>>(in, in_f, in_scale, relu_in, wt, bias, mask, \
                                                                  out, z, x_out, G);                           \
    break;
    CTOF_CONV_CASE(4)
    CTOF_CONV_CASE(2)
    CTOF_CONV_CASE(1)
#undef CTOF_CONV_CASE
  }
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

// relu_out: store ReLU(out) (the next layer applies ReLU to its input, so
// storing it after the ReLU gives that layer the same values).
ctof_status conv_first(const float* z, float in_scale, const __nv_bfloat16* wt, const float* bias,
                       __nv_bfloat16* out, Geo G, bool relu_out, cudaStream_t st) {
  const int txc = G.x % 64 == 0 ? 4 : (G.x % 32 == 0 ? 2 : 1);
  const dim3 grid(G.x / (16 * txc), G.y / CV_TY, G.b * G.z);
#define CTOF_FIRST_CASE(T)                                                                                    \
  if (relu_out)                                                                                               \
    k_conv_first<T, true><<<grid, CV_THREADS, 0, st>>>(z, in_scale, wt, bias, out, G);                      \
  else                                                                                                        \
    k_conv_first<T, false><<<grid, CV_THREADS, 0, st>>>(z, in_scale, wt, bias, out, G);
  if (txc == 4) {
    CTOF_FIRST_CASE(4)
  } else if (txc == 2) {
    CTOF_FIRST_CASE(2)
  } else {
    CTOF_FIRST_CASE(1)
  }
#undef CTOF_FIRST_CASE
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

// Inference hidden / last layer on tcgen05 (input stored after its ReLU):
// out = ReLU(conv(in) + bias), or with prox x_out = z + mu0 bf16(conv(in)[0] + bias[0]).
// EUNSUPPORTED when the activation cannot be described by a tensor map.
ctof_status conv_tc(const ctof_kernel_s* k, const __nv_bfloat16* in, const __nv_bfloat16* wt, const float* bias,
                    __nv_bfloat16* out, const float* z, float* x_out, Geo G, bool prox, cudaStream_t st) {
  CUtensorMap amap;
  const unsigned long long X = G.x, Y = G.y, Z = G.z;
  const unsigned long long dims[5] = {16, X, Y, Z, (unsigned long long)G.b};
  const unsigned long long strides[4] = {32, X * 32, Y * X * 32, Z * Y * X * 32};
  const unsigned box[5] = {16, 130, 1, 1, 1};
  if (ctof_encode_map(&amap, 2, 5, in, dims, strides, box, 32) != CTOF_OK) {
    ctof_set_last_error_text("");
    return CTOF_EUNSUPPORTED;
  }
  const int nunits = G.b * G.z * ((G.y + TCV_YB - 1) / TCV_YB) * ((G.x + 127) / 128);
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, k->device);
  const int grid = nunits < 3 * nsm ? nunits : 3 * nsm;
  if (prox) {
    CTOF_CUDA_TRY(cudaFuncSetAttribute(k_conv3d_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TCV_SMEM));
    k_conv3d_tc<true><<<grid, TCV_THREADS, TCV_SMEM, st>>>(amap, wt, bias, out, z, x_out, G, k->d_flags,
                                                           k->max_polls);
  } else {
    CTOF_CUDA_TRY(
        cudaFuncSetAttribute(k_conv3d_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TCV_SMEM));
    k_conv3d_tc<false><<<grid, TCV_THREADS, TCV_SMEM, st>>>(amap, wt, bias, out, z, x_out, G, k->d_flags,
                                                            k->max_polls);
  }
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

ctof_status conv(const __nv_bfloat16* in, int relu_in, const __nv_bfloat16* wt, const float* bias,
                 const __nv_bfloat16* mask, __nv_bfloat16* out, Geo G, cudaStream_t st) {
  return conv_launch<false, false>(in, nullptr, 0.f, relu_in, wt, bias, mask, out, nullptr, nullptr, G, st);
}

ctof_status wgrad(const __nv_bfloat16* dy, const __nv_bfloat16* x, int relu_in, Geo G, float* part, int nblk, float* acc,
                  cudaStream_t st) {
  k_wgrad<<<nblk, 256, 0, st>>>(dy, x, relu_in, G, part);
  CTOF_CUDA_TRY(cudaGetLastError());
  k_reduce_parts<<<(27 * CH * CH + 255) / 256, 256, 0, st>>>(part, nblk, acc);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

// Operator applications for the whole batch: one contraction launch per
// direction that reads W_hat once for all volumes; lateral FFTs of the depth
// planes as one plane-batched transform (w.inter_zb) or per volume, of the
// time planes per volume.

// T-side spectra of A x for every batch member: w.spec_t [batch][nf][ldt].
ctof_status spectra_forward(ctof_kernel_s* k, int batch, const float* x, const Ws& w, cudaStream_t st) {
  const size_t vol = (size_t)k->nz * k->n * k->n, sz = (size_t)k->nf * k->ldz;
  if (w.inter_zb) {  // all volumes' depth planes as one transform
    CTOF_TRY(fft_forward_planes(k, x, batch * k->nz, k->n, k->n, k->n, w.inter_zb, w.spec_z, w.ldzb, st));
    return contract_tc_forward_zb(k, batch, w.spec_z, w.ldzb, w.spec_t, st);
  }
  for (int b = 0; b < batch; ++b)
    CTOF_TRY(fft_forward_planes(k, x + b * vol, k->nz, k->n, k->n, k->n, k->d_inter_z, w.spec_z + b * sz, k->ldz, st));
  return contract_forward_batch(k, batch, w.spec_z, w.spec_t, st);
}

// out = A^T r (tik_hinv null) or the Tikhonov solve T r = (G + lambda I)^-1 W^T r
// (per frequency), from the T-side spectra of r in w.spec_t.
ctof_status spectra_adjoint(ctof_kernel_s* k, int batch, float* out, const float* tik_hinv, const Ws& w,
                            cudaStream_t st) {
  const size_t vol = (size_t)k->nz * k->n * k->n, sz = (size_t)k->nf * k->ldz;
  if (w.inter_zb) {  // all volumes' depth planes as one transform
    if (tik_hinv)
      CTOF_TRY(contract_tikhonov_zb(k, batch, tik_hinv, w.spec_t, w.spec_z, w.ldzb, st));
    else
      CTOF_TRY(contract_tc_adjoint_zb(k, batch, w.spec_t, w.spec_z, w.ldzb, st));
    return fft_inverse_planes(k, w.spec_z, w.ldzb, batch * k->nz, k->n, k->n, w.inter_zb, out, k->n, st);
  }
  if (tik_hinv)
    CTOF_TRY(contract_tikhonov_batch(k, batch, tik_hinv, w.spec_t, w.spec_z, st));
  else
    CTOF_TRY(contract_adjoint_batch(k, batch, w.spec_t, w.spec_z, st));
  for (int b = 0; b < batch; ++b)
    CTOF_TRY(fft_inverse_planes(k, w.spec_z + b * sz, k->ldz, k->nz, k->n, k->n, k->d_inter_z, out + b * vol, k->n,
                                st));
  return CTOF_OK;
}

// out = A^T r or T r for measurements r [batch][nt][n][n].
ctof_status op_adjoint(ctof_kernel_s* k, int batch, const float* r, float* out, const float* tik_hinv, const Ws& w,
                       cudaStream_t st) {
  const size_t mt = (size_t)k->nt * k->n * k->n, stt = (size_t)k->nf * k->ldt;
  for (int b = 0; b < batch; ++b)
    CTOF_TRY(fft_forward_planes(k, r + b * mt, k->nt, k->n, k->n, k->n, k->d_inter_t, w.spec_t + b * stt, k->ldt, st));
  return spectra_adjoint(k, batch, out, tik_hinv, w, st);
}

// out = A^T (A x - m) (tik_hinv null) or T (A x - m), unnormalised operator, m
// may be null.  The residual never exists in the measurement domain: each
// volume's T side is one inverse column pass of the spectra of A x, one row
// pass that transforms back, crops to the scan, subtracts m and transforms
// forward again, and one forward column pass (Eq. 11 and its adjoint).
ctof_status residual_back(ctof_kernel_s* k, int batch, const float* x, const float* m, float* out,
                          const float* tik_hinv, const Ws& w, cudaStream_t st) {
  const size_t mt = (size_t)k->nt * k->n * k->n, stt = (size_t)k->nf * k->ldt;
  CTOF_TRY(spectra_forward(k, batch, x, w, st));
  for (int b = 0; b < batch; ++b) {
    float2* spec = w.spec_t + b * stt;
    CTOF_TRY(fft_cols_inverse(k, spec, k->ldt, k->nt, k->n, k->d_inter_t, st));
    CTOF_TRY(fft_rows_resid_t(k, k->d_inter_t, m ? m + b * mt : nullptr, st));
    CTOF_TRY(fft_cols_forward(k, k->d_inter_t, k->nt, k->n, spec, k->ldt, st));
  }
  return spectra_adjoint(k, batch, out, tik_hinv, w, st);
}

// Relative data residuals res[b] = ||A x_b - m_b|| / ||m_b|| (FP64 sums of the
// FP32 values), the spectra of A x transformed back one volume at a time and
// compared with m inside the row pass.
ctof_status data_residuals(ctof_kernel_s* k, int batch, const float* x, const float* m, double* res, const Ws& w,
                           cudaStream_t st) {
  const size_t mt = (size_t)k->nt * k->n * k->n, stt = (size_t)k->nf * k->ldt;
  CTOF_CUDA_TRY(cudaMemsetAsync(w.acc, 0, (size_t)batch * 2 * sizeof(double), st));
  CTOF_TRY(spectra_forward(k, batch, x, w, st));
  for (int b = 0; b < batch; ++b) {
    CTOF_TRY(fft_cols_inverse(k, w.spec_t + b * stt, k->ldt, k->nt, k->n, k->d_inter_t, st));
    CTOF_TRY(fft_rows_inverse_norm(k, k->d_inter_t, k->nt, k->n, k->n, m + b * mt, k->n, w.acc + 2 * b, st));
  }
  k_ratio_sqrt<<<(batch + 127) / 128, 128, 0, st>>>(w.acc, batch, res);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

// Forward pass of the unrolled solver; with `train` every stage's activations are kept.
ctof_status unrolled_forward(ctof_learned_s* L, ctof_kernel_s* k, int batch, const float* m, const Ws& w, bool train,
                             cudaStream_t st) {
  const long long V = (long long)batch * k->nz * k->n * k->n;
  const Geo G{batch, k->nz, k->n, k->n};
  const float inv_s2 = (float)(1.0 / (k->scale * k->scale));
  const int nstore = train ? L->stages : 1;
  const float* eta = L->d_theta + L->nparam - L->stages;
  if (L->opt.x0_lambda_rel > 0.0) {
    const float* hinv = nullptr;
    CTOF_TRY(tikhonov_inverse(k, L->opt.x0_lambda_rel * k->gram_max, &hinv, st));
    CTOF_TRY(op_adjoint(k, batch, m, w.x, hinv, w, st));
  } else {
    CTOF_CUDA_TRY(cudaMemsetAsync(w.x, 0, V * sizeof(float), st));
  }
  for (int s = 0; s < L->stages; ++s) {
    const int j = train ? s : 0;
    (void)nstore;
    float* z = w.z + (size_t)j * V;
    float* g = w.g + (size_t)j * V;
    __nv_bfloat16* u = w.u + (size_t)j * V * CH;
    __nv_bfloat16* y1 = w.y1 + (size_t)j * V * CH;
    __nv_bfloat16* y2 = w.y2 + (size_t)j * V * CH;
    __nv_bfloat16* y3 = w.y3 + (size_t)j * V * CH;
    CTOF_TRY(residual_back(k, batch, w.x, m, g, nullptr, w, st));
    k_zstep<<<grid_for(V), 256, 0, st>>>(w.x, g, eta, s, inv_s2, V, z);
    CTOF_CUDA_TRY(cudaGetLastError());
    if (train) {  // the backward pass needs the network input u
      k_pack1<<<grid_for(V), 256, 0, st>>>(z, 1.0f / MU0, V, u);
      CTOF_CUDA_TRY(cudaGetLastError());
      CTOF_TRY(conv(u, 0, L->d_wf + 0 * 27 * CH * CH, L->d_bias + 0 * CH, nullptr, y1, G, st));
    } else {
      // inference: activations stored after their ReLU; hidden and last layers on tcgen05
      CTOF_TRY(conv_first(z, 1.0f / MU0, L->d_wf, L->d_bias, y1, G, true, st));
      const ctof_status s2 = conv_tc(k, y1, L->d_wf + 1 * 27 * CH * CH, L->d_bias + 1 * CH, y2, nullptr, nullptr, G,
                                     false, st);
      if (s2 == CTOF_OK) {
        CTOF_TRY(conv_tc(k, y2, L->d_wf + 2 * 27 * CH * CH, L->d_bias + 2 * CH, y3, nullptr, nullptr, G, false, st));
        CTOF_TRY(conv_tc(k, y3, L->d_wf + 3 * 27 * CH * CH, L->d_bias + 3 * CH, nullptr, z, w.x, G, true, st));
        continue;
      }
      if (s2 != CTOF_EUNSUPPORTED) return s2;
    }
    CTOF_TRY(conv(y1, 1, L->d_wf + 1 * 27 * CH * CH, L->d_bias + 1 * CH, nullptr, y2, G, st));
    CTOF_TRY(conv(y2, 1, L->d_wf + 2 * 27 * CH * CH, L->d_bias + 2 * CH, nullptr, y3, G, st));
    // last layer with the residual step fused: x = z + mu0 f(u)
    CTOF_TRY((conv_launch<false, true>(y3, nullptr, 0.f, 1, L->d_wf + 3 * 27 * CH * CH, L->d_bias + 3 * CH,
                                       nullptr, nullptr, z, w.x, G, st)));
  }
  if (!train && L->opt.dc_steps > 0) {
    // x <- x - T(A x - m): the residual goes through the Tikhonov solve into w.h
    const float* hinv = nullptr;
    CTOF_TRY(tikhonov_inverse(k, L->opt.dc_lambda_rel * k->gram_max, &hinv, st));
    for (int d = 0; d < L->opt.dc_steps; ++d) {
      CTOF_TRY(residual_back(k, batch, w.x, m, w.h, hinv, w, st));
      CTOF_CUDA_TRY(sub_inplace(w.x, w.h, V, st));
    }
  }
  return CTOF_OK;
}

// Loss and flat gradient (accumulated into d_grad, which is zeroed first).
ctof_status unrolled_backward(ctof_learned_s* L, ctof_kernel_s* k, int batch, const float* mu, const Ws& w,
                              cudaStream_t st) {
  const long long V = (long long)batch * k->nz * k->n * k->n;
  const Geo G{batch, k->nz, k->n, k->n};
  const float inv_s2 = (float)(1.0 / (k->scale * k->scale));
  const float* eta = L->d_theta + L->nparam - L->stages;
  float* deta = L->d_grad + L->nparam - L->stages;
  CTOF_CUDA_TRY(cudaMemsetAsync(L->d_grad, 0, L->nparam * sizeof(float), st));
  CTOF_CUDA_TRY(cudaMemsetAsync(L->d_dw, 0, (size_t)NLAYER * 27 * CH * CH * sizeof(float), st));
  CTOF_CUDA_TRY(cudaMemsetAsync(L->d_db, 0, (size_t)NLAYER * CH * sizeof(float), st));
  CTOF_CUDA_TRY(cudaMemsetAsync(L->d_loss, 0, sizeof(double), st));
  k_loss<<<grid_for(V), 256, 0, st>>>(w.x, mu, V, w.gx, L->d_loss);
  CTOF_CUDA_TRY(cudaGetLastError());
  const int bg_blocks = grid_for(V) < 304 ? grid_for(V) : 304;
  for (int s = L->stages - 1; s >= 0; --s) {
    const float* g = w.g + (size_t)s * V;
    const __nv_bfloat16* u = w.u + (size_t)s * V * CH;
    const __nv_bfloat16* y1 = w.y1 + (size_t)s * V * CH;
    const __nv_bfloat16* y2 = w.y2 + (size_t)s * V * CH;
    const __nv_bfloat16* y3 = w.y3 + (size_t)s * V * CH;
    // x_{s+1} = z + mu0 f(u): output gradient of f is mu0 * gx
    k_pack1<<<grid_for(V), 256, 0, st>>>(w.gx, MU0, V, w.da);
    CTOF_CUDA_TRY(cudaGetLastError());
    const __nv_bfloat16* acts[NLAYER] = {u, y1, y2, y3};
    const __nv_bfloat16* pre[NLAYER] = {nullptr, y1, y2, y3};
    __nv_bfloat16* cur = w.da;
    __nv_bfloat16* nxt = w.db_;
    for (int l = NLAYER - 1; l >= 0; --l) {
      CTOF_TRY(wgrad(cur, acts[l], l > 0 ? 1 : 0, G, w.part, w.nblk, L->d_dw + (size_t)l * 27 * CH * CH, st));
      k_bias_grad<<<bg_blocks, 256, 0, st>>>(cur, V, L->d_db + l * CH);
      CTOF_CUDA_TRY(cudaGetLastError());
      // gradient w.r.t. this layer's input: masked by the ReLU of the previous pre-activation
      CTOF_TRY(conv(cur, 0, L->d_wb + (size_t)l * 27 * CH * CH, nullptr, pre[l], nxt, G, st));
      __nv_bfloat16* t = cur;
      cur = nxt;
      nxt = t;
    }
    // cur holds dL/du (channel 0); z = x - eta g,  g = A_n^T (A_n x - m_n)
    k_gz<<<grid_for(V) < 304 ? grid_for(V) : 304, 256, 0, st>>>(w.gx, cur, g, V, w.gz, deta, s);
    CTOF_CUDA_TRY(cudaGetLastError());
    CTOF_TRY(residual_back(k, batch, w.gz, nullptr, w.h, nullptr, w, st));
    k_gx<<<grid_for(V), 256, 0, st>>>(w.gz, w.h, eta, s, inv_s2, V, w.gx);
    CTOF_CUDA_TRY(cudaGetLastError());
  }
  for (int l = 0; l < NLAYER; ++l) {
    const int n = L->lo[l].co * L->lo[l].ci * 27;
    k_grad_to_flat<<<(n + 255) / 256, 256, 0, st>>>(L->d_dw + (size_t)l * 27 * CH * CH, L->d_db + l * CH, L->lo[l],
                                                    L->d_grad);
    CTOF_CUDA_TRY(cudaGetLastError());
  }
  return CTOF_OK;
}

ctof_status check_geometry(const ctof_kernel_s* k) {
  if (k->n % 16 != 0) return CTOF_EUNSUPPORTED;  // convolution tiles are 16 voxels along x
  return CTOF_OK;
}

}  // namespace

extern "C" {

int ctof_learned_param_count(int stages) {
  int n = 0;
  for (int l = 0; l < NLAYER; ++l) n += LAYER_OUT[l] * LAYER_IN[l] * 27 + LAYER_OUT[l];
  return n + stages;
}

ctof_status ctof_learned_create(int stages, const float* h_params, const ctof_learned_options* opt,
                                ctof_learned* out) {
  if (!out || !h_params || stages < 1 || stages > 64) return CTOF_EINVAL;
  ctof_learned_options o{};
  if (opt) o = *opt;
  if (!(o.x0_lambda_rel >= 0.0) || !isfinite(o.x0_lambda_rel) || o.dc_steps < 0 || o.dc_steps > 16 ||
      (o.dc_steps > 0 && !(o.dc_lambda_rel > 0.0 && isfinite(o.dc_lambda_rel))))
    return CTOF_EINVAL;
  *out = nullptr;
  ctof_learned_s* L = new (std::nothrow) ctof_learned_s();
  if (!L) return CTOF_ENOMEM;
  L->stages = stages;
  L->nparam = ctof_learned_param_count(stages);
  L->opt = o;
  CTOF_CUDA_TRY(cudaGetDevice(&L->device));
  int off = 0;
  for (int l = 0; l < NLAYER; ++l) {
    L->lo[l].ci = LAYER_IN[l];
    L->lo[l].co = LAYER_OUT[l];
    L->lo[l].w = off;
    off += LAYER_OUT[l] * LAYER_IN[l] * 27;
    L->lo[l].b = off;
    off += LAYER_OUT[l];
  }
  const size_t np = L->nparam;
  const size_t bytes = 4 * np * 4 + 2 * (size_t)NLAYER * 27 * CH * CH * 2 + (size_t)NLAYER * CH * 4 +
                       (size_t)NLAYER * 27 * CH * CH * 4 + (size_t)NLAYER * CH * 4 + 64;
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete L;
    return CTOF_ENOMEM;
  }
  char* b = static_cast<char*>(p);
  L->d_theta = reinterpret_cast<float*>(b);
  L->d_grad = L->d_theta + np;
  L->d_m1 = L->d_grad + np;
  L->d_m2 = L->d_m1 + np;
  L->d_wf = reinterpret_cast<__nv_bfloat16*>(L->d_m2 + np);
  L->d_wb = L->d_wf + (size_t)NLAYER * 27 * CH * CH;
  L->d_bias = reinterpret_cast<float*>(L->d_wb + (size_t)NLAYER * 27 * CH * CH);
  L->d_dw = L->d_bias + NLAYER * CH;
  L->d_db = L->d_dw + (size_t)NLAYER * 27 * CH * CH;
  L->d_loss = reinterpret_cast<double*>(reinterpret_cast<uintptr_t>(L->d_db + NLAYER * CH + 8) & ~(uintptr_t)7);
  if (cudaMemcpy(L->d_theta, h_params, np * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(L->d_m1, 0, 2 * np * 4) != cudaSuccess || learned_prep(L, nullptr) != CTOF_OK ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaFree(p);
    delete L;
    return CTOF_ECUDA;
  }
  *out = L;
  return CTOF_OK;
}

void ctof_learned_destroy(ctof_learned L) {
  if (!L) return;
  if (L->d_ws) cudaFree(L->d_ws);
  cudaFree(L->d_theta);
  delete L;
}

ctof_status ctof_learned_get_params(ctof_learned L, float* h_params) {
  if (!L || !h_params) return CTOF_EINVAL;
  CTOF_CUDA_TRY(cudaMemcpy(h_params, L->d_theta, (size_t)L->nparam * 4, cudaMemcpyDeviceToHost));
  return CTOF_OK;
}

ctof_status ctof_learned_loss_grad(ctof_learned L, ctof_kernel k, int batch, const float* d_m, const float* d_mu,
                                   double* h_loss, float* h_grad, void* stream) {
  if (!L || !k || !d_m || !d_mu || batch < 1) return CTOF_EINVAL;
  CTOF_TRY(check_geometry(k));
  if (L->device != k->device) return CTOF_EINVAL;
  DeviceGuard dg(k->device);
  if (!dg.ok) return CTOF_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Ws w;
  CTOF_TRY(learned_workspace(L, k, batch, true, &w));
  CTOF_TRY(unrolled_forward(L, k, batch, d_m, w, true, st));
  CTOF_TRY(unrolled_backward(L, k, batch, d_mu, w, st));
  double loss = 0.0;
  CTOF_CUDA_TRY(cudaMemcpyAsync(&loss, L->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (h_grad) CTOF_CUDA_TRY(cudaMemcpyAsync(h_grad, L->d_grad, (size_t)L->nparam * 4, cudaMemcpyDeviceToHost, st));
  const ctof_status waits = take_device_status(k, st);  // synchronises
  const long long V = (long long)batch * k->nz * k->n * k->n;
  if (h_loss) *h_loss = loss / (double)V;
  return waits;
}

ctof_status ctof_learned_train_step(ctof_learned L, ctof_kernel k, int batch, const float* d_m, const float* d_mu,
                                    double lr, double* h_loss, void* stream) {
  if (!L || !k || !d_m || !d_mu || batch < 1 || !(lr > 0)) return CTOF_EINVAL;
  CTOF_TRY(check_geometry(k));
  if (L->device != k->device) return CTOF_EINVAL;
  DeviceGuard dg(k->device);
  if (!dg.ok) return CTOF_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Ws w;
  CTOF_TRY(learned_workspace(L, k, batch, true, &w));
  CTOF_TRY(unrolled_forward(L, k, batch, d_m, w, true, st));
  CTOF_TRY(unrolled_backward(L, k, batch, d_mu, w, st));
  L->adam_step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)L->adam_step), c2 = 1.f - powf(b2, (float)L->adam_step);
  k_adam<<<(L->nparam + 255) / 256, 256, 0, st>>>(L->d_theta, L->d_grad, L->d_m1, L->d_m2, L->nparam, (float)lr, b1, b2,
                                                  1e-8f, c1, c2);
  CTOF_CUDA_TRY(cudaGetLastError());
  CTOF_TRY(learned_prep(L, st));
  if (h_loss) {
    double loss = 0.0;
    CTOF_CUDA_TRY(cudaMemcpyAsync(&loss, L->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    const ctof_status waits = take_device_status(k, st);  // synchronises
    *h_loss = loss / (double)((long long)batch * k->nz * k->n * k->n);
    return waits;
  }
  return CTOF_OK;
}

ctof_status ctof_learned_reconstruct(ctof_learned L, ctof_kernel k, int batch, const float* d_m, float* d_mu,
                                     void* stream) {
  if (!L || !k || !d_m || !d_mu || batch < 1) return CTOF_EINVAL;
  CTOF_TRY(check_geometry(k));
  if (L->device != k->device) return CTOF_EINVAL;
  DeviceGuard dg(k->device);
  if (!dg.ok) return CTOF_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Ws w;
  CTOF_TRY(learned_workspace(L, k, batch, false, &w));
  CTOF_TRY(unrolled_forward(L, k, batch, d_m, w, false, st));
  CTOF_CUDA_TRY(cudaMemcpyAsync(d_mu, w.x, (size_t)batch * k->nz * k->n * k->n * 4, cudaMemcpyDeviceToDevice, st));
  return CTOF_OK;
}

ctof_status ctof_learned_reconstruct_checked(ctof_learned L, ctof_kernel k, int batch, const float* d_m,
                                             float* d_mu, double* d_res, void* stream) {
  if (!L || !k || !d_m || !d_mu || !d_res || batch < 1) return CTOF_EINVAL;
  CTOF_TRY(check_geometry(k));
  if (L->device != k->device) return CTOF_EINVAL;
  DeviceGuard dg(k->device);
  if (!dg.ok) return CTOF_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Ws w;
  CTOF_TRY(learned_workspace(L, k, batch, false, &w));
  CTOF_TRY(unrolled_forward(L, k, batch, d_m, w, false, st));
  CTOF_TRY(data_residuals(k, batch, w.x, d_m, d_res, w, st));
  CTOF_CUDA_TRY(cudaMemcpyAsync(d_mu, w.x, (size_t)batch * k->nz * k->n * k->n * 4, cudaMemcpyDeviceToDevice, st));
  return CTOF_OK;
}

}  // extern "C"
