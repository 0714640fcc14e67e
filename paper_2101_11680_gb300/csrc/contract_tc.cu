// Batched per-frequency contractions on the 5th-generation tensor cores
// (tcgen05, TMEM accumulators): the forward M_hat(f, t) = sum_z W_hat(f, t, z)
// mu_hat(f, z) and the adjoint V_hat(f, z) = sum_t W_hat(f, t, z) r_hat(f, t)
// of Eq. 11 in the lateral Fourier domain, for many volumes that share one
// kernel.  A frequency class (up to 4 frequencies with the same real T x Z
// block) and 16 volumes give 16 x 4 x 2 = 128 real right-hand sides, so each
// class is one GEMM with a 128-wide side:
//   forward  D[t][n] = sum_z W[t][z] X[n][z]   M = 128 rows of t, N = 128, K = z
//   adjoint  D[n][z] = sum_t C[n][t] W[t][z]   M = 128,  N = Z (to 16), K = t
// (n = 8 v + 2 m + c: volume v of the chunk, member m, real/imaginary c).
// Operands are staged in shared memory in the no-swizzle K-major layout of
// umma.cuh, each split into a TF32 high part and an FP32 remainder; three
// MMAs per K step (lo*hi + hi*lo + hi*hi) keep FP32-level accuracy.  The
// adjoint's W^T is formed by the staging itself (4 x 4 register transposes),
// so W_hat is read from its one [class][t][z] table.  One elected thread issues
// the MMAs and commits them to an mbarrier; the CTA waits on it with a
// bounded poll (a timeout sets the handle's timeout flag), then every warp
// reads its 32-lane quarter of TMEM for the epilogue.  Persistent CTAs walk
// the classes; two fit on an SM when their shared memory allows, so one
// CTA's staging overlaps the other's MMAs and stores.
// A wait that runs out (after the handle's poll limit) sets the handle's
// sticky status flag, waits again with the fixed drain limit so that no MMA
// is left in flight, and the whole CTA then stops (a block-wide vote), frees
// its TMEM and returns; the host reports CTOF_ETIMEOUT at the next
// synchronising call.
#include <cuda_runtime.h>

#include "bulk.cuh"
#include "ctof_internal.h"
#include "umma.cuh"

namespace {

constexpr int TC_THREADS = 256;
constexpr int VB = 16;         // volumes per chunk
constexpr int NR = 8 * VB;     // right-hand sides per chunk (the 128-wide GEMM side)
constexpr int TCH = 32;        // adjoint: t values per staged K chunk
constexpr int RCS = TCH * 8 + 16;  // adjoint raw stage: bytes per (volume, member) row, padded
constexpr long long DRAIN_POLLS = 1ll << 24;  // polls of the wait that follows a timeout

struct TcPlan {
  int nt, nz, z4, zK, zN, tK, tc;
  int off_ahi, off_alo, off_bhi, off_blo, off_bar, total;
  int off_raw, raw_c, raw_stage;  // adjoint: two raw stages of [64 rows][RCS] C and [tc][z4] W
  uint32_t ncols;  // TMEM columns
};

inline int rup(int x, int m) { return (x + m - 1) / m * m; }

// Forward: A = W rows (128 per M tile) x zK, B = X rows (128) x zK.
TcPlan plan_fwd(int nt, int nz) {
  TcPlan p{};
  p.nt = nt;
  p.nz = nz;
  p.z4 = rup(nz, 4);
  p.zK = rup(nz, 8);
  const int tile = 128 * p.zK * 4;
  p.off_ahi = 0;
  p.off_alo = tile;
  p.off_bhi = 2 * tile;
  p.off_blo = 3 * tile;
  p.off_bar = 4 * tile;
  p.total = p.off_bar + 64;
  p.ncols = 128;
  return p;
}

// Adjoint: A = C rows (128) x tc, B = W^T rows (zN) x tc, per K chunk of tc t values.
TcPlan plan_adj(int nt, int nz) {
  TcPlan p{};
  p.nt = nt;
  p.nz = nz;
  p.z4 = rup(nz, 4);
  p.zN = rup(nz, 16);
  p.tK = rup(nt, 8);
  p.tc = p.tK < TCH ? p.tK : TCH;
  const int ta = 128 * p.tc * 4, tb = p.zN * p.tc * 4;
  p.off_ahi = 0;
  p.off_alo = ta;
  p.off_bhi = 2 * ta;
  p.off_blo = 2 * ta + tb;
  p.raw_c = 4 * VB * RCS;
  p.raw_stage = p.raw_c + p.tc * p.z4 * 4;
  p.off_raw = 2 * ta + 2 * tb;
  p.off_bar = p.off_raw + 2 * p.raw_stage;
  p.total = p.off_bar + 64;
  p.ncols = p.zN <= 32 ? 32 : 64;
  return p;
}

__device__ __forceinline__ void st_split4(unsigned char* sm, const TcPlan& P, uint32_t off, float4 v) {
  float4 h, l;
  umma::split_tf32(v.x, h.x, l.x);
  umma::split_tf32(v.y, h.y, l.y);
  umma::split_tf32(v.z, h.z, l.z);
  umma::split_tf32(v.w, h.w, l.w);
  *reinterpret_cast<float4*>(sm + P.off_ahi + off) = h;
  *reinterpret_cast<float4*>(sm + P.off_alo + off) = l;
}

// mem[m] for a runtime m without spilling the array to local memory
__device__ __forceinline__ int pick(const int (&mem)[4], int m) {
  return m == 0 ? mem[0] : (m == 1 ? mem[1] : (m == 2 ? mem[2] : mem[3]));
}

__device__ __forceinline__ void st_split1(unsigned char* hi, unsigned char* lo, uint32_t off, float v) {
  float h, l;
  umma::split_tf32(v, h, l);
  *reinterpret_cast<float*>(hi + off) = h;
  *reinterpret_cast<float*>(lo + off) = l;
}

// Setup shared by both kernels: zero shared memory (padding rows and columns
// of the operand tiles stay zero), allocate TMEM, initialise the mbarrier.
__device__ __forceinline__ uint32_t tc_setup(unsigned char* sm, const TcPlan& P) {
  for (int i = threadIdx.x; i < P.total / 16; i += blockDim.x)
    reinterpret_cast<float4*>(sm)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + P.off_bar);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + P.off_bar + 16);
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) umma::tmem_alloc(slot, P.ncols);
  if (threadIdx.x == 0) umma::mbar_init(bar, 1);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  return *slot;
}

__device__ __forceinline__ void tc_teardown(uint32_t taddr, const TcPlan& P) {
  umma::fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) umma::tmem_dealloc(taddr, P.ncols);
}

// Staged operands -> visible to the tensor core; all threads.
__device__ __forceinline__ void publish() {
  umma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
}

// Wait for the committed MMAs (phase parity).  After max_polls polls the
// wait gives up: it sets the timeout flag and drains (waits up to
// DRAIN_POLLS more for the MMAs in flight).  Block-wide: returns true when
// any thread of the CTA gave up, and then the CTA must stop.
__device__ __forceinline__ bool wait_mma(uint64_t* bar, uint32_t& phase, int* timeout_flag, long long max_polls) {
  int gave_up = 0;
  if (!umma::mbar_wait(bar, phase, max_polls)) {
    gave_up = 1;
    atomicExch(timeout_flag, 1);
    umma::mbar_wait(bar, phase, DRAIN_POLLS);
  }
  phase ^= 1u;
  umma::fence_after_sync();
  return __syncthreads_or(gave_up) != 0;
}

__global__ void __launch_bounds__(TC_THREADS, 2) k_contract_tc_fwd(TcPlan P, const float* __restrict__ what,
                                                               const int* __restrict__ members, int nclass, int nvol,
                                                               const float2* __restrict__ vin, int ld_in,
                                                               size_t in_vstride, float2* __restrict__ vout,
                                                               int ld_out, size_t out_vstride, int* timeout_flag,
                                                               long long max_polls) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const uint32_t taddr = tc_setup(sm, P);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + P.off_bar);
  uint32_t phase = 0;
  bool stop = false;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nt = P.nt, nz = P.nz, q4 = P.z4 >> 2;
  const uint32_t idesc = umma::idesc_tf32(128, NR);
  const uint32_t sbase = umma::smem_u32(sm);
  for (int c = blockIdx.x; c < nclass && !stop; c += gridDim.x) {
    int mem[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) mem[m] = __ldg(members + 4 * c + m);
    const float* wc = what + (size_t)c * nt * P.z4;
    for (int v0 = 0; v0 < nvol && !stop; v0 += VB) {
      const int nv = nvol - v0 < VB ? nvol - v0 : VB;
      // B: X[n][z] for the chunk's volumes (rows of absent members are zero).
      // A warp takes 8 (volume, member) rows x 4 chunks of 4 complex z: 128
      // contiguous bytes per row on the load side, consecutive rows on the
      // store side.  All loads are issued before the first store.
      const int nvm = nv * 4, zq = (nz + 3) >> 2, kgb = (zq + 3) >> 2, nbb = ((nvm + 7) >> 3) * kgb;
      {
        float4 x[4][2];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int blk = u * (TC_THREADS / 32) + warp, rg = blk / kgb, kg = blk - rg * kgb;
          const int vm = 8 * rg + (lane & 7), zc = 4 * kg + (lane >> 3);
          x[u][0] = x[u][1] = make_float4(0.f, 0.f, 0.f, 0.f);
          const int f = vm < nvm ? pick(mem, vm & 3) : -1;
          if (blk < nbb && vm < nvm && zc < zq && f >= 0) {
            const float2* src = vin + (v0 + (vm >> 2)) * in_vstride + (size_t)f * ld_in + 4 * zc;
            if (4 * zc + 4 <= nz) {
              x[u][0] = __ldg(reinterpret_cast<const float4*>(src));
              x[u][1] = __ldg(reinterpret_cast<const float4*>(src) + 1);
            } else {
              float e[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
              for (int q = 0; q < 4 && 4 * zc + q < nz; ++q) {
                const float2 y = src[q];
                e[2 * q] = y.x;
                e[2 * q + 1] = y.y;
              }
              x[u][0] = make_float4(e[0], e[1], e[2], e[3]);
              x[u][1] = make_float4(e[4], e[5], e[6], e[7]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int blk = u * (TC_THREADS / 32) + warp, rg = blk / kgb, kg = blk - rg * kgb;
          const int vm = 8 * rg + (lane & 7), zc = 4 * kg + (lane >> 3);
          if (blk < nbb && vm < nvm && zc < zq) {
            const float4 re = make_float4(x[u][0].x, x[u][0].z, x[u][1].x, x[u][1].z);
            const float4 im = make_float4(x[u][0].y, x[u][0].w, x[u][1].y, x[u][1].w);
            float4 h, l;
            umma::split_tf32(re.x, h.x, l.x);
            umma::split_tf32(re.y, h.y, l.y);
            umma::split_tf32(re.z, h.z, l.z);
            umma::split_tf32(re.w, h.w, l.w);
            *reinterpret_cast<float4*>(sm + P.off_bhi + umma::kmajor_off(NR, 2 * vm, 4 * zc)) = h;
            *reinterpret_cast<float4*>(sm + P.off_blo + umma::kmajor_off(NR, 2 * vm, 4 * zc)) = l;
            umma::split_tf32(im.x, h.x, l.x);
            umma::split_tf32(im.y, h.y, l.y);
            umma::split_tf32(im.z, h.z, l.z);
            umma::split_tf32(im.w, h.w, l.w);
            *reinterpret_cast<float4*>(sm + P.off_bhi + umma::kmajor_off(NR, 2 * vm + 1, 4 * zc)) = h;
            *reinterpret_cast<float4*>(sm + P.off_blo + umma::kmajor_off(NR, 2 * vm + 1, 4 * zc)) = l;
          }
        }
      }
      for (int t0 = 0; t0 < nt; t0 += 128) {
        const int rows = nt - t0 < 128 ? nt - t0 : 128;
        // A: W rows t0 .. t0 + rows.  A warp takes 8 rows x 4 float4 chunks
        // (64 contiguous bytes per row to load, 8 consecutive 16-byte tile rows
        // per store phase); at most 16 x 4 blocks, 8 per warp; loads first.
        const int kga = (q4 + 3) >> 2, nba = ((rows + 7) >> 3) * kga;
        float4 w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int blk = u * (TC_THREADS / 32) + warp, rg = blk / kga, kg = blk - rg * kga;
          const int tl = 8 * rg + (lane & 7), k4 = 4 * kg + (lane >> 3);
          if (blk < nba && tl < rows && k4 < q4)
            w[u] = __ldg(reinterpret_cast<const float4*>(wc + (size_t)(t0 + tl) * P.z4) + k4);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int blk = u * (TC_THREADS / 32) + warp, rg = blk / kga, kg = blk - rg * kga;
          const int tl = 8 * rg + (lane & 7), k4 = 4 * kg + (lane >> 3);
          if (blk < nba && tl < rows && k4 < q4) st_split4(sm, P, umma::kmajor_off(128, tl, 4 * k4), w[u]);
        }
        publish();
        if (tid == 0) {
          for (int s = 0; s < P.zK / 8; ++s) {
            const uint32_t o = s * 2 * 128 * 16;
            const uint64_t ah = umma::desc(sbase + P.off_ahi + o, 128 * 16, 128);
            const uint64_t al = umma::desc(sbase + P.off_alo + o, 128 * 16, 128);
            const uint64_t bh = umma::desc(sbase + P.off_bhi + o, NR * 16, 128);
            const uint64_t bl = umma::desc(sbase + P.off_blo + o, NR * 16, 128);
            umma::mma_tf32(taddr, al, bh, idesc, s > 0);
            umma::mma_tf32(taddr, ah, bl, idesc, 1);
            umma::mma_tf32(taddr, ah, bh, idesc, 1);
          }
          umma::commit(bar);
        }
        if (wait_mma(bar, phase, timeout_flag, max_polls)) {
          stop = true;
          break;
        }
        // epilogue: TMEM lane = t row of the tile; warps w and w + 4 split the 8 column groups
        const int tl = 32 * (warp & 3) + lane, t = t0 + tl;
        for (int j = warp >> 2; j < NR / 16; j += 2) {
          float d[16];
          umma::tmem_ld16(taddr + ((uint32_t)(32 * (warp & 3)) << 16) + 16 * j, d);
#pragma unroll
          for (int vv = 0; vv < 2; ++vv) {
            const int v = 2 * j + vv;
            if (v < nv && t < nt) {
#pragma unroll
              for (int m = 0; m < 4; ++m)
                if (mem[m] >= 0)
                  vout[(v0 + v) * out_vstride + (size_t)mem[m] * ld_out + t] =
                      make_float2(d[8 * vv + 2 * m], d[8 * vv + 2 * m + 1]);
            }
          }
        }
        umma::fence_before_sync();
        __syncthreads();
      }
    }
  }
  tc_teardown(taddr, P);
}

// Adjoint.  The CTA's steps are s = (class, volume chunk, t chunk).  Step
// s + 1's input rows (64 (volume, member) rows of TCH complex t values, and
// TCH rows of W) stream into the other of two raw shared-memory stages with
// coalesced 16-byte cp.async copies while step s is converted (raw -> split
// K-major tiles, W transposed through 4 x 4 register blocks) and multiplied.
struct AdjStep {
  int c, v0, nv, t0, tcc, last;
};

__device__ __forceinline__ AdjStep adj_step(const TcPlan& P, int s, int nvol, int nvc, int ntc) {
  AdjStep a;
  const int per = nvc * ntc, j = s / per, r = s - j * per, vc = r / ntc, tci = r - vc * ntc;
  a.c = blockIdx.x + j * gridDim.x;
  a.v0 = vc * VB;
  a.nv = nvol - a.v0 < VB ? nvol - a.v0 : VB;
  a.t0 = tci * P.tc;
  a.tcc = P.tK - a.t0 < P.tc ? P.tK - a.t0 : P.tc;
  a.last = tci == ntc - 1;
  return a;
}

__device__ __forceinline__ void load_members(const int* __restrict__ members, int c, int (&mem)[4]) {
#pragma unroll
  for (int m = 0; m < 4; ++m) mem[m] = __ldg(members + 4 * c + m);
}

// 16-byte asynchronous copy; bytes < 16 zero-fills the rest (0: no read)
__device__ __forceinline__ void cp_async16z(void* smem, const void* gmem, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(umma::smem_u32(smem)), "l"(gmem),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ void adj_issue(const TcPlan& P, unsigned char* sm, int stage, const AdjStep& a,
                                          const int (&mem)[4], const float* __restrict__ what,
                                          const float2* __restrict__ vin, int ld_in, size_t in_vstride) {
  unsigned char* rc = sm + P.off_raw + stage * P.raw_stage;
  unsigned char* rw = rc + P.raw_c;
  const int nt = P.nt, q4 = P.z4 >> 2, pieces = a.tcc >> 1, nvm = a.nv * 4;
  // (row, piece) of copy i = tid + k * TC_THREADS, advanced without divisions
  {
    int vm = threadIdx.x / pieces, p = threadIdx.x - vm * pieces;
    const int dvm = TC_THREADS / pieces, dp = TC_THREADS - dvm * pieces;
    while (vm < nvm) {
      const int f = pick(mem, vm & 3), t = a.t0 + 2 * p;
      const int bytes = f < 0 ? 0 : (t + 2 <= nt ? 16 : (t < nt ? 8 : 0));
      const float2* src = bytes ? vin + (a.v0 + (vm >> 2)) * in_vstride + (size_t)f * ld_in + t : vin;
      cp_async16z(rc + vm * RCS + p * 16, src, bytes);
      vm += dvm;
      p += dp;
      if (p >= pieces) {
        p -= pieces;
        ++vm;
      }
    }
  }
  const float* wc = what + (size_t)a.c * nt * P.z4;
  {
    int tl = threadIdx.x / q4, k4 = threadIdx.x - tl * q4;
    const int dtl = TC_THREADS / q4, dk = TC_THREADS - dtl * q4;
    while (tl < a.tcc) {
      const int t = a.t0 + tl, bytes = t < nt ? 16 : 0;
      cp_async16z(rw + (tl * q4 + k4) * 16, bytes ? wc + (size_t)t * P.z4 + 4 * k4 : what, bytes);
      tl += dtl;
      k4 += dk;
      if (k4 >= q4) {
        k4 -= q4;
        ++tl;
      }
    }
  }
}

__device__ __forceinline__ void adj_convert(const TcPlan& P, unsigned char* sm, int stage, const AdjStep& a) {
  const unsigned char* rc = sm + P.off_raw + stage * P.raw_stage;
  const unsigned char* rw = rc + P.raw_c;
  const int q4 = P.z4 >> 2, nvm = a.nv * 4, t4n = a.tcc >> 2;
  // A: C[n][t] from the raw rows; consecutive threads on consecutive rows
  {
    int t4 = threadIdx.x / nvm, vm = threadIdx.x - t4 * nvm;
    const int dt = TC_THREADS / nvm, dv = TC_THREADS - dt * nvm;
    while (t4 < t4n) {
      const float4* r = reinterpret_cast<const float4*>(rc + vm * RCS + t4 * 32);
      const float4 x0 = r[0], x1 = r[1];
      st_split4(sm, P, umma::kmajor_off(NR, 2 * vm, 4 * t4), make_float4(x0.x, x0.z, x1.x, x1.z));
      st_split4(sm, P, umma::kmajor_off(NR, 2 * vm + 1, 4 * t4), make_float4(x0.y, x0.w, x1.y, x1.w));
      t4 += dt;
      vm += dv;
      if (vm >= nvm) {
        vm -= nvm;
        ++t4;
      }
    }
  }
  // B: W^T[z][t] from 4 x 4 blocks of the raw W rows, transposed in registers
  for (int i = threadIdx.x; i < t4n * q4; i += TC_THREADS) {
    const int t4 = i / q4, k4 = i - t4 * q4;
    float4 w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) w[e] = *reinterpret_cast<const float4*>(rw + ((4 * t4 + e) * q4 + k4) * 16);
    const float col[4][4] = {{w[0].x, w[1].x, w[2].x, w[3].x},
                             {w[0].y, w[1].y, w[2].y, w[3].y},
                             {w[0].z, w[1].z, w[2].z, w[3].z},
                             {w[0].w, w[1].w, w[2].w, w[3].w}};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      float4 h, l;
      umma::split_tf32(col[r][0], h.x, l.x);
      umma::split_tf32(col[r][1], h.y, l.y);
      umma::split_tf32(col[r][2], h.z, l.z);
      umma::split_tf32(col[r][3], h.w, l.w);
      const uint32_t o = umma::kmajor_off(P.zN, 4 * k4 + r, 4 * t4);
      *reinterpret_cast<float4*>(sm + P.off_bhi + o) = h;
      *reinterpret_cast<float4*>(sm + P.off_blo + o) = l;
    }
  }
}

__global__ void __launch_bounds__(TC_THREADS, 2) k_contract_tc_adj(TcPlan P, const float* __restrict__ what,
                                                               const int* __restrict__ members, int nclass, int nvol,
                                                               const float2* __restrict__ vin, int ld_in,
                                                               size_t in_vstride, float2* __restrict__ vout,
                                                               int ld_out, size_t out_vstride, int* timeout_flag,
                                                               long long max_polls) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const uint32_t taddr = tc_setup(sm, P);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + P.off_bar);
  uint32_t phase = 0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t idesc = umma::idesc_tf32(128, P.zN);
  const uint32_t sbase = umma::smem_u32(sm);
  const int nvc = (nvol + VB - 1) / VB, ntc = (P.tK + P.tc - 1) / P.tc;
  const int mine = blockIdx.x < nclass ? (nclass - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int steps = mine * nvc * ntc;
  int mem[4], mem_next[4];
  if (steps > 0) {
    const AdjStep a0 = adj_step(P, 0, nvol, nvc, ntc);
    load_members(members, a0.c, mem_next);
    adj_issue(P, sm, 0, a0, mem_next, what, vin, ld_in, in_vstride);
  }
  cp_commit();
  for (int s = 0; s < steps; ++s) {
    const AdjStep a = adj_step(P, s, nvol, nvc, ntc);
#pragma unroll
    for (int m = 0; m < 4; ++m) mem[m] = mem_next[m];
    if (s + 1 < steps) {  // the other raw stage was last read by step s - 1's conversion
      const AdjStep b = adj_step(P, s + 1, nvol, nvc, ntc);
      if (b.c != a.c) load_members(members, b.c, mem_next);
      adj_issue(P, sm, (s + 1) & 1, b, mem_next, what, vin, ld_in, in_vstride);
    }
    cp_commit();
    cp_wait1();  // every group but the newest: step s's copies have landed
    __syncthreads();
    adj_convert(P, sm, s & 1, a);
    publish();
    if (tid == 0) {
      for (int k = 0; k < a.tcc / 8; ++k) {
        const uint64_t ah = umma::desc(sbase + P.off_ahi + k * 2 * NR * 16, NR * 16, 128);
        const uint64_t al = umma::desc(sbase + P.off_alo + k * 2 * NR * 16, NR * 16, 128);
        const uint64_t bh = umma::desc(sbase + P.off_bhi + k * 2 * P.zN * 16, P.zN * 16, 128);
        const uint64_t bl = umma::desc(sbase + P.off_blo + k * 2 * P.zN * 16, P.zN * 16, 128);
        umma::mma_tf32(taddr, al, bh, idesc, (a.t0 > 0 || k > 0) ? 1u : 0u);
        umma::mma_tf32(taddr, ah, bl, idesc, 1);
        umma::mma_tf32(taddr, ah, bh, idesc, 1);
      }
      umma::commit(bar);
    }
    if (wait_mma(bar, phase, timeout_flag, max_polls)) break;
    if (a.last) {
      // epilogue: TMEM lane n = 8 v + 2 m + c; column z.  Even lanes hold the
      // real parts, odd lanes the imaginary parts of the same output.
      const int n = 32 * (warp & 3) + lane, v = n >> 3, fm = pick(mem, (n >> 1) & 3);
      const bool writer = (lane & 1) == 0 && v < a.nv && fm >= 0;
      float2* dst = vout + (a.v0 + (v < a.nv ? v : 0)) * out_vstride + (size_t)(fm >= 0 ? fm : 0) * ld_out;
      for (int j = warp >> 2; j < P.zN / 16; j += 2) {
        float d[16];
        umma::tmem_ld16(taddr + ((uint32_t)(32 * (warp & 3)) << 16) + 16 * j, d);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const float im = __shfl_down_sync(0xffffffffu, d[e], 1);
          const int z = 16 * j + e;
          if (writer && z < P.nz) dst[z] = make_float2(d[e], im);
        }
      }
    }
    // the next step's publish() orders these TMEM reads before its MMAs
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  tc_teardown(taddr, P);
}

// ---- warp-specialised adjoint (bins a multiple of 16) ----
//
// D[n][z] = sum_t C[n][t] W[t][z] for (class, 16-volume chunk) items, with
// n = 32 m + 16 c + v (member, real / imaginary, volume).  Warp 0 (one
// thread) stages each chunk of 32 t with tensor-map copies (per member one
// box of 2 halves x 16 volumes x 16 t of r_hat [v][f][t], two W_hat boxes of
// 32 t x 32 z; 128-byte swizzle) into AW_STAGES raw stages; warps 1-8 split a
// staged chunk into TF32 high parts and FP32 remainders in the K-major
// layout (as many term sets as raw stages); warp 9 (one thread) issues three
// MMAs per K = 8 step into one of two TMEM accumulators; warps 12-15 write
// the finished item out.  mbarrier hand-offs; every wait is bounded, a wait
// that runs out sets the handle's flag and a shared abort word and every
// role leaves its loop.
constexpr int AW_CONV = 8;
constexpr int AW_MMA_WARP = 9;
constexpr int AW_EPI0 = 12;
constexpr int AW_THREADS = (AW_EPI0 + 4) * 32;
constexpr int AW_STAGES = 3;
constexpr int AW_MBOX = 16 * 16 * 8;  // r_hat box of one member and one 16-t half
constexpr int AW_WBOX = 32 * 32 * 4;  // W_hat box: 32 t x 32 z

struct AwPlan {
  int nt, nz, z4, zn, nwb;
  int a_term, b_term, set_bytes, raw_stage;
  int off_raw, off_set, off_bar, total;
};

AwPlan make_aw_plan(int nt, int nz) {
  AwPlan P{};
  P.nt = nt;
  P.nz = nz;
  P.z4 = rup(nz, 4);
  P.zn = rup(nz, 16);
  P.nwb = P.z4 <= 32 ? 1 : 2;
  P.a_term = NR * TCH * 4;
  P.b_term = P.zn * TCH * 4;
  P.set_bytes = 2 * (P.a_term + P.b_term);
  P.raw_stage = rup(8 * AW_MBOX + P.nwb * AW_WBOX, 1024);
  P.off_raw = 0;
  P.off_set = AW_STAGES * P.raw_stage;
  P.off_bar = P.off_set + AW_STAGES * P.set_bytes;
  P.total = P.off_bar + 256 + 1024;  // + room to align the base to 1024 bytes
  return P;
}

__device__ __forceinline__ bool aw_wait(uint64_t* bar, uint32_t parity, long long max_polls, volatile int* abort_w,
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

__device__ __forceinline__ bool aw_wait_warp(uint64_t* bar, uint32_t parity, long long max_polls,
                                             volatile int* abort_w, int* flag, int lane) {
  int ok = 1;
  if (lane == 0) ok = aw_wait(bar, parity, max_polls, abort_w, flag) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok && lane != 0) (void)bulk::try_wait(bar, parity);
  return ok != 0;
}

// Split one staged chunk (converter thread ct of 256): A rows n (K = t) and
// B = W^T rows z (K = t), TF32 high part and FP32 remainder each.
__device__ __forceinline__ void aw_convert(const AwPlan& P, const unsigned char* raw, unsigned char* set,
                                           const int (&mem)[4], int ct) {
  unsigned char* ahi = set;
  unsigned char* alo = set + P.a_term;
  unsigned char* bhi = set + 2 * P.a_term;
  unsigned char* blo = bhi + P.b_term;
  for (int i = ct; i < 64 * (TCH / 4); i += AW_CONV * 32) {
    const int v = i & 15, m = (i >> 4) & 3, gI = i >> 6;  // 4 t values 4 gI ..
    const int nre = 32 * m + v, nim = nre + 16;
    const uint32_t o_re = umma::kmajor_off(NR, nre, 4 * gI), o_im = umma::kmajor_off(NR, nim, 4 * gI);
    float4 re = make_float4(0.f, 0.f, 0.f, 0.f), im = re;
    if (pick(mem, m) >= 0) {
      const int t0 = 4 * gI;
      const unsigned char* rowp = raw + (2 * m + (t0 >> 4)) * AW_MBOX + v * 128;
      const int c0 = (t0 & 15) >> 1;
      const float4 q0 = *reinterpret_cast<const float4*>(rowp + ((c0 ^ (v & 7)) << 4));
      const float4 q1 = *reinterpret_cast<const float4*>(rowp + (((c0 + 1) ^ (v & 7)) << 4));
      re = make_float4(q0.x, q0.z, q1.x, q1.z);
      im = make_float4(q0.y, q0.w, q1.y, q1.w);
    }
    float4 h, l;
    umma::split_tf32(re.x, h.x, l.x);
    umma::split_tf32(re.y, h.y, l.y);
    umma::split_tf32(re.z, h.z, l.z);
    umma::split_tf32(re.w, h.w, l.w);
    *reinterpret_cast<float4*>(ahi + o_re) = h;
    *reinterpret_cast<float4*>(alo + o_re) = l;
    umma::split_tf32(im.x, h.x, l.x);
    umma::split_tf32(im.y, h.y, l.y);
    umma::split_tf32(im.z, h.z, l.z);
    umma::split_tf32(im.w, h.w, l.w);
    *reinterpret_cast<float4*>(ahi + o_im) = h;
    *reinterpret_cast<float4*>(alo + o_im) = l;
  }
  const unsigned char* rw = raw + 8 * AW_MBOX;
  for (int i = ct; i < P.zn * (TCH / 4); i += AW_CONV * 32) {
    const int z = i % P.zn, gI = i / P.zn;
    const unsigned char* box = rw + (z >> 5) * AW_WBOX + (z & 3) * 4;
    const int zc = (z & 31) >> 2;
    float w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int t = 4 * gI + e;
      w[e] = *reinterpret_cast<const float*>(box + t * 128 + ((zc ^ (t & 7)) << 4));
    }
    float4 h, l;
    umma::split_tf32(w[0], h.x, l.x);
    umma::split_tf32(w[1], h.y, l.y);
    umma::split_tf32(w[2], h.z, l.z);
    umma::split_tf32(w[3], h.w, l.w);
    const uint32_t o = umma::kmajor_off(P.zn, z, 4 * gI);
    *reinterpret_cast<float4*>(bhi + o) = h;
    *reinterpret_cast<float4*>(blo + o) = l;
  }
}

__global__ void __launch_bounds__(AW_THREADS, 1)
    k_contract_tc_adj_ws(const __grid_constant__ CUtensorMap cmap, const __grid_constant__ CUtensorMap wmap,
                         AwPlan P, const int* __restrict__ members, int nclass, int nvol,
                         float2* __restrict__ vout, int ld_out, size_t out_vstride, int* flag, long long max_polls) {
  extern __shared__ float4 aw_smem4[];
  unsigned char* sm;
  {
    const uint32_t s = bulk::saddr(aw_smem4);
    sm = reinterpret_cast<unsigned char*>(aw_smem4) + (((s + 1023u) & ~1023u) - s);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nt = P.nt, nz = P.nz, zn = P.zn;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + P.off_bar);
  uint64_t* raw_full = bar;                       // [S] one arrival + the copies' bytes
  uint64_t* raw_empty = bar + AW_STAGES;          // [S] one arrival per converter warp
  uint64_t* term_full = bar + 2 * AW_STAGES;      // [S] one arrival per converter warp
  uint64_t* term_empty = bar + 3 * AW_STAGES;     // [S] the MMAs that read the set (commit)
  uint64_t* acc_full = bar + 4 * AW_STAGES;       // [2] the item's MMAs (commit)
  uint64_t* acc_empty = acc_full + 2;             // [2] one arrival per epilogue warp
  uint64_t* drain_bar = acc_empty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain_bar + 1);
  volatile int* abort_w = reinterpret_cast<volatile int*>(drain_bar + 2);
  if (threadIdx.x == 0) {
    for (int i = 0; i < AW_STAGES; ++i) {
      bulk::bar_init(raw_full + i, 1);
      bulk::bar_init(raw_empty + i, AW_CONV);
      bulk::bar_init(term_full + i, AW_CONV);
      bulk::bar_init(term_empty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      bulk::bar_init(acc_full + i, 1);
      bulk::bar_init(acc_empty + i, 4);
    }
    bulk::bar_init(drain_bar, 1);
    *abort_w = 0;
  }
  if (warp == 0) umma::tmem_alloc(tslot, 128);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t taddr = *tslot;
  const int nchunks = (nt + TCH - 1) / TCH, nvc = (nvol + VB - 1) / VB;

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int gk = 0;
      bool ok = true;
      for (int c = blockIdx.x; c < nclass && ok; c += gridDim.x) {
        int mem[4];
        int present = 0;
        for (int m = 0; m < 4; ++m) {
          mem[m] = __ldg(members + 4 * c + m);
          present += mem[m] >= 0;
        }
        for (int vc = 0; vc < nvc && ok; ++vc)
          for (int kc = 0; kc < nchunks; ++kc, ++gk) {
            const int s = gk % AW_STAGES;
            if (gk >= AW_STAGES &&
                !aw_wait(raw_empty + s, (uint32_t)((gk / AW_STAGES) + 1) & 1u, max_polls, abort_w, flag)) {
              ok = false;
              break;
            }
            unsigned char* st = sm + P.off_raw + s * P.raw_stage;
            bulk::arrive_expect(raw_full + s, (unsigned)(present * 2 * AW_MBOX + P.nwb * AW_WBOX));
            for (int m = 0; m < 4; ++m)
              if (mem[m] >= 0)
                bulk::tensor_g2s_4d(st + 2 * m * AW_MBOX, &cmap, 0, vc * VB, 2 * kc, mem[m], raw_full + s);
            for (int wb = 0; wb < P.nwb; ++wb)
              bulk::tensor_g2s_2d(st + 8 * AW_MBOX + wb * AW_WBOX, &wmap, 32 * wb, c * nt + kc * TCH, raw_full + s);
          }
      }
      for (int s = 0; s < AW_STAGES && s < gk; ++s)
        bulk::wait(raw_full + s, (uint32_t)((gk - 1 - s) / AW_STAGES) & 1u, DRAIN_POLLS);
    }
  } else if (warp <= AW_CONV) {
    // ---------------- converters ----------------
    const int ct = threadIdx.x - 32;
    int gk = 0;
    bool ok = true;
    for (int c = blockIdx.x; c < nclass && ok; c += gridDim.x) {
      int mem[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) mem[m] = __ldg(members + 4 * c + m);
      for (int vc = 0; vc < nvc && ok; ++vc)
        for (int kc = 0; kc < nchunks; ++kc, ++gk) {
          const int s = gk % AW_STAGES;
          if (!aw_wait_warp(raw_full + s, (uint32_t)(gk / AW_STAGES) & 1u, max_polls, abort_w, flag, lane) ||
              (gk >= AW_STAGES && !aw_wait_warp(term_empty + s, (uint32_t)((gk / AW_STAGES) + 1) & 1u, max_polls,
                                                abort_w, flag, lane))) {
            ok = false;
            break;
          }
          aw_convert(P, sm + P.off_raw + s * P.raw_stage, sm + P.off_set + s * P.set_bytes, mem, ct);
          umma::fence_proxy_async();  // this lane's term writes, before the MMAs read them
          __syncwarp();
          if (lane == 0) {
            bulk::arrive(raw_empty + s);
            bulk::arrive(term_full + s);
          }
        }
    }
  } else if (warp == AW_MMA_WARP) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = umma::idesc_tf32(NR, zn);
      const uint32_t sbase = bulk::saddr(sm);
      int gk = 0, it = 0;
      bool ok = true;
      for (int c = blockIdx.x; c < nclass && ok; c += gridDim.x)
        for (int vc = 0; vc < nvc && ok; ++vc, ++it) {
          const int a = it & 1;
          if (it >= 2 && !aw_wait(acc_empty + a, (uint32_t)((it >> 1) + 1) & 1u, max_polls, abort_w, flag)) {
            ok = false;
            break;
          }
          umma::fence_after_sync();
          const uint32_t acc = taddr + (uint32_t)(a * 64);
          for (int kc = 0; kc < nchunks; ++kc, ++gk) {
            const int s = gk % AW_STAGES;
            if (!aw_wait(term_full + s, (uint32_t)(gk / AW_STAGES) & 1u, max_polls, abort_w, flag)) {
              ok = false;
              break;
            }
            umma::fence_after_sync();
            const uint32_t a0 = sbase + P.off_set + s * P.set_bytes;
            const uint32_t b0 = a0 + 2 * P.a_term;
            for (int k = 0; k < TCH / 8; ++k) {
              const uint64_t ah = umma::desc(a0 + k * 2 * NR * 16, NR * 16, 128);
              const uint64_t al = umma::desc(a0 + P.a_term + k * 2 * NR * 16, NR * 16, 128);
              const uint64_t bh = umma::desc(b0 + k * 2 * zn * 16, zn * 16, 128);
              const uint64_t bl = umma::desc(b0 + P.b_term + k * 2 * zn * 16, zn * 16, 128);
              umma::mma_tf32(acc, al, bh, idesc, (kc > 0 || k > 0) ? 1u : 0u);
              umma::mma_tf32(acc, ah, bl, idesc, 1);
              umma::mma_tf32(acc, ah, bh, idesc, 1);
            }
            umma::commit(term_empty + s);
          }
          if (ok) umma::commit(acc_full + a);
        }
      umma::commit(drain_bar);
      bulk::wait(drain_bar, 0, DRAIN_POLLS);
    }
  } else if (warp >= AW_EPI0) {
    // ---------------- epilogue: write the item's D ----------------
    const int n = 32 * (warp & 3) + lane;  // TMEM lane = right-hand side
    const uint32_t trow = taddr + ((uint32_t)(32 * (warp & 3)) << 16);
    const int v = n & 15, ri = (n >> 4) & 1, m = n >> 5;
    int it = 0;
    bool ok = true;
    for (int c = blockIdx.x; c < nclass && ok; c += gridDim.x) {
      int mem[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) mem[q] = __ldg(members + 4 * c + q);
      for (int vc = 0; vc < nvc && ok; ++vc, ++it) {
        const int a = it & 1, v0 = vc * VB, nv = nvol - v0 < VB ? nvol - v0 : VB;
        if (!aw_wait_warp(acc_full + a, (uint32_t)(it >> 1) & 1u, max_polls, abort_w, flag, lane)) {
          ok = false;
          break;
        }
        umma::fence_after_sync();
        const int fm = pick(mem, m);
        const bool writer = ri == 0 && v < nv && fm >= 0;
        float2* dst = vout + (size_t)(v0 + (v < nv ? v : 0)) * out_vstride + (size_t)(fm >= 0 ? fm : 0) * ld_out;
        for (int j = 0; j < zn / 16; ++j) {
          float d[16];
          umma::tmem_ld16(trow + (uint32_t)(a * 64 + 16 * j), d);
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const float im = __shfl_down_sync(0xffffffffu, d[e], 16);
            const int z = 16 * j + e;
            if (writer && z < nz) dst[z] = make_float2(d[e], im);
          }
        }
        umma::fence_before_sync();
        __syncwarp();
        if (lane == 0) bulk::arrive(acc_empty + a);
      }
    }
  }
  __syncwarp();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (warp == 0) umma::tmem_dealloc(taddr, 128);
}

template <typename K>
ctof_status launch_tc(K kern, const TcPlan& P, const ctof_kernel_s* k, int nvol, const float2* vin, int ld_in,
                      size_t in_vstride, float2* vout, int ld_out, size_t out_vstride, cudaStream_t st) {
  if (P.total > 227 * 1024) return CTOF_EUNSUPPORTED;
  CTOF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, P.total));
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, k->device);
  // resident CTAs per SM: shared memory, registers (65,536 per SM, allocated
  // in units of 8 per thread) and TMEM (512 columns per SM), at most 4; the
  // persistent grid is exactly that many CTAs per SM
  int per_sm = (228 * 1024) / (P.total + 1024);
  cudaFuncAttributes fa;
  CTOF_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
  const int regs = (fa.numRegs + 7) / 8 * 8 * TC_THREADS;
  if (regs > 0 && 65536 / regs < per_sm) per_sm = 65536 / regs;
  const int tmem_cap = (int)(512 / P.ncols);
  if (per_sm > 4) per_sm = 4;
  if (per_sm > tmem_cap) per_sm = tmem_cap;
  if (per_sm < 1) per_sm = 1;
  const int grid = k->nclass < per_sm * nsm ? k->nclass : per_sm * nsm;
  kern<<<grid, TC_THREADS, P.total, st>>>(P, k->d_what, k->d_members, k->nclass, nvol, vin, ld_in, in_vstride, vout,
                                          ld_out, out_vstride, k->d_flags, k->max_polls);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

// The warp-specialised adjoint when the bins are a multiple of 16 (tensor-map
// staging) and its buffers take tensor maps; EUNSUPPORTED otherwise.
ctof_status launch_adj_ws(const ctof_kernel_s* k, int nvol, const float2* vin, int ld_in, size_t in_vstride,
                          float2* vout, int ld_out, size_t out_vstride, cudaStream_t st) {
  if (k->nt % 16 != 0 || rup(k->nz, 16) > 64) return CTOF_EUNSUPPORTED;
  const AwPlan P = make_aw_plan(k->nt, k->nz);
  if (P.total > 227 * 1024) return CTOF_EUNSUPPORTED;
  CUtensorMap cmap, wmap;
  // r_hat element (t = 16 h + tt, v, f) as a 4-D tensor (tt, v, h, f)
  const unsigned long long cdims[4] = {16, (unsigned long long)nvol, (unsigned long long)k->nt / 16,
                                       (unsigned long long)k->nf};
  const unsigned long long cstr[3] = {(unsigned long long)in_vstride * 8, 16 * 8, (unsigned long long)ld_in * 8};
  const unsigned cbox[4] = {16, VB, 2, 1};
  const unsigned long long wdims[2] = {(unsigned long long)k->z4, (unsigned long long)k->nt * k->nclass};
  const unsigned long long wstr[1] = {(unsigned long long)k->z4 * 4};
  const unsigned wbox[2] = {32, TCH};
  if (ctof_encode_map(&cmap, 8, 4, vin, cdims, cstr, cbox, 128) != CTOF_OK ||
      ctof_encode_map(&wmap, 4, 2, k->d_what, wdims, wstr, wbox, 128) != CTOF_OK) {
    ctof_set_last_error_text("");
    return CTOF_EUNSUPPORTED;
  }
  CTOF_CUDA_TRY(cudaFuncSetAttribute(k_contract_tc_adj_ws, cudaFuncAttributeMaxDynamicSharedMemorySize, P.total));
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, k->device);
  const int grid = k->nclass < nsm ? k->nclass : nsm;
  k_contract_tc_adj_ws<<<grid, AW_THREADS, P.total, st>>>(cmap, wmap, P, k->d_members, k->nclass, nvol, vout, ld_out,
                                                          out_vstride, k->d_flags, k->max_polls);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

}  // namespace

ctof_status contract_tc_forward(const ctof_kernel_s* k, int nvol, const float2* in_z, float2* out_t,
                                cudaStream_t st) {
  if (nvol < 1) return CTOF_EINVAL;
  return launch_tc(k_contract_tc_fwd, plan_fwd(k->nt, k->nz), k, nvol, in_z, k->ldz, (size_t)k->nf * k->ldz, out_t,
                   k->ldt, (size_t)k->nf * k->ldt, st);
}

ctof_status contract_tc_adjoint(const ctof_kernel_s* k, int nvol, const float2* in_t, float2* out_z,
                                cudaStream_t st) {
  if (nvol < 1) return CTOF_EINVAL;
  const ctof_status s =
      launch_adj_ws(k, nvol, in_t, k->ldt, (size_t)k->nf * k->ldt, out_z, k->ldz, (size_t)k->nf * k->ldz, st);
  if (s != CTOF_EUNSUPPORTED) return s;
  return launch_tc(k_contract_tc_adj, plan_adj(k->nt, k->nz), k, nvol, in_t, k->ldt, (size_t)k->nf * k->ldt, out_z,
                   k->ldz, (size_t)k->nf * k->ldz, st);
}

ctof_status contract_tc_forward_zb(const ctof_kernel_s* k, int nvol, const float2* in_z, int ldzb, float2* out_t,
                                   cudaStream_t st) {
  if (nvol < 1 || (k->nz & 1) || (ldzb & 7) || ldzb < nvol * k->nz) return CTOF_EINVAL;
  return launch_tc(k_contract_tc_fwd, plan_fwd(k->nt, k->nz), k, nvol, in_z, ldzb, (size_t)k->nz, out_t, k->ldt,
                   (size_t)k->nf * k->ldt, st);
}

ctof_status contract_tc_adjoint_zb(const ctof_kernel_s* k, int nvol, const float2* in_t, float2* out_z, int ldzb,
                                   cudaStream_t st) {
  if (nvol < 1 || (k->nz & 1) || (ldzb & 7) || ldzb < nvol * k->nz) return CTOF_EINVAL;
  const ctof_status s = launch_adj_ws(k, nvol, in_t, k->ldt, (size_t)k->nf * k->ldt, out_z, ldzb, (size_t)k->nz, st);
  if (s != CTOF_EUNSUPPORTED) return s;
  return launch_tc(k_contract_tc_adj, plan_adj(k->nt, k->nz), k, nvol, in_t, k->ldt, (size_t)k->nf * k->ldt, out_z,
                   ldzb, (size_t)k->nz, st);
}
