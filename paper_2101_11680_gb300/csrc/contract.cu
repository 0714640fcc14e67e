// Per-frequency contractions of the convolutional model (Eq. 11 in the
// lateral Fourier domain): for every half-plane frequency f,
//   forward   M_hat(f, t) = sum_z W_hat(f, t, z) mu_hat(f, z)       (T x Z . Z)
//   adjoint   V_hat(f, z) = sum_t W_hat(f, t, z) r_hat(f, t)        (Z x T . T)
//   Tikhonov  x_hat(f)    = (G(f) + lambda I)^-1 V_hat(f)           (Z x Z)
// W_hat is real (the kernel is even in x and y) and, for dx == dy, equal on
// the up-to-four frequencies (a,b), (a,-b), (b,a), (b,-a) of one class, so
// each class's T x Z block is read from HBM once and applied to the complex
// vectors of all members (up to 8 real right-hand sides).
//
// Persistent CTAs walk the classes with a two-stage cp.async pipeline: while
// one class is computed, the next class's W_hat block (contiguous in HBM,
// rows of z4 floats) and, for Tikhonov, its FP64 inverse stream into the other
// shared-memory stage.  A launch may carry several volumes that share the
// kernel (`nvol`, spectra `vstride` apart): the class block then stays in
// shared memory while the volumes' member vectors stream through their own
// double buffer, so W_hat is read once for all of them.  W_hat rows land with a stride
// of 4*(z4/4 | 1) floats, so eight consecutive rows read with float4 loads hit
// eight distinct 16-byte bank groups.  The arithmetic is FP32 FMA: these
// contractions move 1 FLOP per 2 bytes of W_hat.  The Tikhonov inverse is
// formed in FP64 and applied in FP32: its rounding error, eps |H^-1| |b|, is
// of the same size as the one b already carries from its FP32 sums.
// (The fused ADMM x-update lives in contract_admm.cu.)
#include <cuda_runtime.h>

#include "ctof_internal.h"

namespace {

constexpr int CT_THREADS = 256;

enum { MODE_FWD = 0, MODE_ADJ = 1, MODE_TIK = 2 };

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async8(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Shared-memory plan: nbuf W stages (W_hat block, Tikhonov inverse), nvs
// vector stages, then the per-CTA scratch.
struct Plan {
  int nt, nz, z4, q, sw;   // q = z4/4 float4 chunks per row, sw = smem row stride (floats)
  int J;                   // adjoint: row groups
  size_t off_h;            // Tikhonov inverse inside a W stage
  size_t wst, vst;         // bytes per W stage / vector stage
  size_t off_v;            // first vector stage
  size_t off_part, off_b;  // scratch
  size_t total;
};

__host__ __device__ inline size_t al16(size_t b) { return (b + 15) & ~(size_t)15; }

__host__ __device__ inline Plan make_plan(int mode, int nt, int nz, int nbuf, int nvs, int threads) {
  Plan p;
  p.nt = nt;
  p.nz = nz;
  p.z4 = (nz + 3) & ~3;
  p.q = p.z4 / 4;
  p.sw = 4 * (p.q | 1);
  const int pairs = 2 * p.q;
  p.J = threads / pairs > 0 ? threads / pairs : 1;
  p.off_h = al16((size_t)nt * p.sw * 4);
  p.wst = p.off_h + (mode == MODE_TIK ? al16((size_t)nz * p.z4 * 4) : 0);
  p.vst = al16(mode == MODE_FWD ? (size_t)p.z4 * 8 * 4 : (size_t)nt * 8 * 4);
  p.off_v = p.wst * nbuf;
  size_t s = p.off_v + p.vst * nvs;
  p.off_part = s;
  if (mode != MODE_FWD) s += al16((size_t)p.J * p.z4 * 8 * 4);
  p.off_b = s;
  if (mode == MODE_TIK) s += al16((size_t)p.z4 * 8 * 4);
  p.total = s;
  return p;
}

// Copies of class c's W_hat block (and Tikhonov inverse) into a W stage.
template <int MODE>
__device__ __forceinline__ void issue_w(const Plan& P, char* stg, int* s_mem, const float* __restrict__ what,
                                        const int* __restrict__ members, const float* __restrict__ hinv, int c) {
  float* sW = reinterpret_cast<float*>(stg);
  const float* src = what + (size_t)c * P.nt * P.z4;
  const int chunks = P.nt * P.q;
  for (int i = threadIdx.x; i < chunks; i += blockDim.x) {
    const int t = i / P.q, k = i - t * P.q;
    cp_async16(sW + t * P.sw + 4 * k, src + (size_t)t * P.z4 + 4 * k);
  }
  if (threadIdx.x < 4) s_mem[threadIdx.x] = members[c * 4 + threadIdx.x];
  if (MODE == MODE_TIK) {
    float* sH = reinterpret_cast<float*>(stg + P.off_h);
    const float* hs = hinv + (size_t)c * P.nz * P.z4;
    for (int i = threadIdx.x; i < P.nz * P.q; i += blockDim.x) cp_async16(sH + 4 * i, hs + 4 * i);
  }
}

// Copies of class c's member vectors of one volume into a vector stage: [row][4] complex.
template <int MODE>
__device__ __forceinline__ void issue_v(const Plan& P, char* vst, const int* __restrict__ members,
                                        const float2* __restrict__ vin, int ld_in, int c) {
  float2* sV = reinterpret_cast<float2*>(vst);
  const int rows = MODE == MODE_FWD ? P.z4 : P.nt;
  const int valid = MODE == MODE_FWD ? P.nz : P.nt;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int f = members[c * 4 + m];
    const float2* src = vin + (size_t)(f < 0 ? 0 : f) * ld_in;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
      if (f >= 0 && r < valid)
        cp_async8(sV + r * 4 + m, src + r);
      else
        sV[r * 4 + m] = make_float2(0.f, 0.f);
    }
  }
}

// out[t][0..7] = sum_z W[t][z] x[z][0..7]  (one thread per row t)
__device__ __forceinline__ void compute_fwd(const Plan& P, const float* sW, const char* sv, const int* s_mem,
                                            float2* __restrict__ out_t, int ldt) {
  const float4* sX = reinterpret_cast<const float4*>(sv);  // [z][2] float4
  for (int t = threadIdx.x; t < P.nt; t += blockDim.x) {
    float acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = 0.f;
    const float4* wr = reinterpret_cast<const float4*>(sW + t * P.sw);
    for (int k = 0; k < P.q; ++k) {
      const float4 w = wr[k];
      const float wz[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 a = sX[(4 * k + j) * 2], b = sX[(4 * k + j) * 2 + 1];
        acc[0] = fmaf(wz[j], a.x, acc[0]);
        acc[1] = fmaf(wz[j], a.y, acc[1]);
        acc[2] = fmaf(wz[j], a.z, acc[2]);
        acc[3] = fmaf(wz[j], a.w, acc[3]);
        acc[4] = fmaf(wz[j], b.x, acc[4]);
        acc[5] = fmaf(wz[j], b.y, acc[5]);
        acc[6] = fmaf(wz[j], b.z, acc[6]);
        acc[7] = fmaf(wz[j], b.w, acc[7]);
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m)
      if (s_mem[m] >= 0) out_t[(size_t)s_mem[m] * ldt + t] = make_float2(acc[2 * m], acc[2 * m + 1]);
  }
}

// Adjoint partial sums: thread (j, k, h) sums rows t = j (mod J) for z in chunk k
// and right-hand sides 4h..4h+3; partials land in part[j][z][8].
__device__ __forceinline__ void compute_adj_partials(const Plan& P, const float* sW, const char* sv, float* part) {
  const float* sC = reinterpret_cast<const float*>(sv);  // [t][8]
  const int pairs = 2 * P.q;
  for (int u = threadIdx.x; u < P.J * pairs; u += blockDim.x) {
    const int j = u / pairs, pk = u - j * pairs, k = pk >> 1, h = pk & 1;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int t = j; t < P.nt; t += P.J) {
      const float4 w = *reinterpret_cast<const float4*>(sW + t * P.sw + 4 * k);
      const float4 cv = *reinterpret_cast<const float4*>(sC + t * 8 + 4 * h);
      const float wz[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        acc[a][0] = fmaf(wz[a], cv.x, acc[a][0]);
        acc[a][1] = fmaf(wz[a], cv.y, acc[a][1]);
        acc[a][2] = fmaf(wz[a], cv.z, acc[a][2]);
        acc[a][3] = fmaf(wz[a], cv.w, acc[a][3]);
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
      *reinterpret_cast<float4*>(part + ((size_t)j * P.z4 + 4 * k + a) * 8 + 4 * h) =
          make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
  }
}

// Steps s = 0, 1, ... of a CTA are (class blockIdx.x + (s / nvol) * gridDim.x,
// volume s % nvol).  The member vectors of step s + nvs - 1 are issued while
// step s computes (one commit group per step).  With two W stages (nbw == 2)
// a class's W_hat block goes with the vectors of its first volume, at most one
// class ahead since nvs <= nvol + 1.  With one W stage (nbw == 1; used when
// many volumes share a class, so that two CTAs fit on an SM) the block is
// loaded when its class starts.  With nvs == 1 nothing overlaps.
template <int MODE>
__device__ __forceinline__ void issue_step(const Plan& P, char* smem, int (*s_mem)[4], const float* __restrict__ what,
                                           const int* __restrict__ members, const float2* __restrict__ vin,
                                           int ld_in, size_t in_vstride, const float* __restrict__ hinv,
                                           int nclass, int nvol, int nbw, int nvs, int s, bool with_w) {
  const int ci = s / nvol, b = s - ci * nvol;
  const int c = blockIdx.x + ci * gridDim.x;
  if (c >= nclass) return;
  const int wb = nbw == 2 ? (ci & 1) : 0;
  if (b == 0 && with_w) issue_w<MODE>(P, smem + wb * P.wst, s_mem[wb], what, members, hinv, c);
  issue_v<MODE>(P, smem + P.off_v + (s % nvs) * P.vst, members, vin + (size_t)b * in_vstride, ld_in, c);
}

template <int MODE>
__global__ void __launch_bounds__(CT_THREADS) k_contract(const float* __restrict__ what,
                                                         const int* __restrict__ members, int nclass, int nt, int nz,
                                                         const float2* __restrict__ vin, int ld_in, size_t in_vstride,
                                                         float2* __restrict__ vout, int ld_out, size_t out_vstride,
                                                         int nvol, const float* __restrict__ hinv, int nbw, int nvs) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int s_mem[2][4];
  const Plan P = make_plan(MODE, nt, nz, nbw, nvs, blockDim.x);
  float* part = reinterpret_cast<float*>(smem + P.off_part);
  float* sB = reinterpret_cast<float*>(smem + P.off_b);
  const int G = gridDim.x;
  const int my_classes = blockIdx.x < nclass ? (nclass - 1 - blockIdx.x) / G + 1 : 0;
  const int nsteps = my_classes * nvol;
  const int ahead = nvs - 1;
  for (int s = 0; s < (ahead > 0 ? ahead : 1); ++s) {
    if (s < nsteps)
      issue_step<MODE>(P, smem, s_mem, what, members, vin, ld_in, in_vstride, hinv, nclass, nvol, nbw, nvs, s,
                       nbw == 2 || s == 0);
    cp_commit();
  }
  for (int s = 0; s < nsteps; ++s) {
    const int ci = s / nvol, b = s - ci * nvol;
    const int wcur = nbw == 2 ? (ci & 1) : 0;
    const int vcur = s % nvs;
    const bool w_now = nbw == 1 && ahead > 0 && b == 0 && s > 0;  // one W stage: load this class now
    if (w_now) issue_w<MODE>(P, smem, s_mem[0], what, members, hinv, blockIdx.x + ci * G);
    if (ahead > 0) {
      if (s + ahead < nsteps)
        issue_step<MODE>(P, smem, s_mem, what, members, vin, ld_in, in_vstride, hinv, nclass, nvol, nbw, nvs,
                         s + ahead, nbw == 2);
      cp_commit();
      // all groups but the newest `ahead` are complete: those hold steps s+1 .. s+ahead
      if (w_now) {
        cp_wait<0>();
      } else {
        switch (ahead) {
          case 1: cp_wait<1>(); break;
          case 2: cp_wait<2>(); break;
          default: cp_wait<3>(); break;
        }
      }
    } else {
      cp_commit();
      cp_wait<0>();
    }
    __syncthreads();
    const char* wst = smem + wcur * P.wst;
    const float* sW = reinterpret_cast<const float*>(wst);
    const char* sv = smem + P.off_v + vcur * P.vst;
    const int* mem = s_mem[wcur];
    float2* out = vout + (size_t)b * out_vstride;
    if (MODE == MODE_FWD) {
      compute_fwd(P, sW, sv, mem, out, ld_out);
    } else {
      compute_adj_partials(P, sW, sv, part);
      __syncthreads();
      if (MODE == MODE_ADJ) {
        for (int o = threadIdx.x; o < 4 * nz; o += blockDim.x) {
          const int m = o / nz, z = o - m * nz;
          if (mem[m] < 0) continue;
          float re = 0.f, im = 0.f;
          for (int j = 0; j < P.J; ++j) {
            re += part[((size_t)j * P.z4 + z) * 8 + 2 * m];
            im += part[((size_t)j * P.z4 + z) * 8 + 2 * m + 1];
          }
          out[(size_t)mem[m] * ld_out + z] = make_float2(re, im);
        }
      } else {
        for (int o = threadIdx.x; o < nz * 8; o += blockDim.x) {
          const int z = o >> 3, r = o & 7;
          float s = 0.f;
          for (int j = 0; j < P.J; ++j) s += part[((size_t)j * P.z4 + z) * 8 + r];
          sB[z * 8 + r] = s;
        }
        __syncthreads();
        // x[i] = sum_j Hinv[j][i] b[j]  (Hinv symmetric; consecutive threads read consecutive i)
        const float* sH = reinterpret_cast<const float*>(wst + P.off_h);
        for (int o = threadIdx.x; o < 4 * nz; o += blockDim.x) {
          const int m = o / nz, i = o - m * nz;
          if (mem[m] < 0) continue;
          float re = 0.f, im = 0.f;
          for (int j = 0; j < nz; ++j) {
            const float h = sH[j * P.z4 + i];
            re = fmaf(h, sB[j * 8 + 2 * m], re);
            im = fmaf(h, sB[j * 8 + 2 * m + 1], im);
          }
          out[(size_t)mem[m] * ld_out + i] = make_float2(re, im);
        }
      }
    }
    __syncthreads();
    if (ahead == 0 && s + 1 < nsteps)
      issue_step<MODE>(P, smem, s_mem, what, members, vin, ld_in, in_vstride, hinv, nclass, nvol, nbw, nvs, s + 1,
                       true);
  }
  cp_wait<0>();
}

constexpr size_t SMEM_LIMIT = 227 * 1024;

// In-place application of the per-class Tikhonov inverse to batched adjoint
// results: x[v][f][i] = sum_j Hinv_c[j][i] x[v][f][j] for every member f of
// class c and volume v (Hinv symmetric, FP32, formed in FP64).  A CTA stages
// the class's inverse and up to 16 volumes' member vectors in shared memory,
// then each thread accumulates a 4 x 4 block (4 consecutive outputs i of 4
// member vectors) in registers: per j one 16-byte read of the inverse row and
// four 8-byte vector reads feed 32 FMAs.  Vector rows are padded to nz + 1
// entries so that the three vector groups a warp reads fall on distinct banks.
constexpr int HV = 16;  // volumes per staged chunk

__global__ void __launch_bounds__(256, 4) k_apply_hinv(const float* __restrict__ hinv,
                                                       const int* __restrict__ members, int nclass, int nz, int z4,
                                                       int nvol, float2* __restrict__ x, int ldz, size_t vstride) {
  extern __shared__ __align__(16) float hsm[];
  const int nzp = nz + 1;
  float* sH = hsm;                                          // [nz][z4], columns nz..z4-1 zero
  float2* sV = reinterpret_cast<float2*>(hsm + nz * z4);    // [HV * 4][nzp]
  const int nig = z4 >> 2;
  for (int c = blockIdx.x; c < nclass; c += gridDim.x) {
    const int4 mem = __ldg(reinterpret_cast<const int4*>(members) + c);
    auto member = [&](int q) { return q == 0 ? mem.x : q == 1 ? mem.y : q == 2 ? mem.z : mem.w; };
    __syncthreads();  // the previous class's reads of sH / sV are done
    for (int i = threadIdx.x; i < nz * z4; i += blockDim.x) sH[i] = __ldg(hinv + (size_t)c * nz * z4 + i);
    for (int v0 = 0; v0 < nvol; v0 += HV) {
      const int nv = nvol - v0 < HV ? nvol - v0 : HV;
      const int R = nv * 4;
      for (int o = threadIdx.x; o < R * nz; o += blockDim.x) {
        const int r = o / nz, j = o - r * nz, f = member(r & 3);
        sV[r * nzp + j] = f >= 0 ? x[(v0 + (r >> 2)) * vstride + (size_t)f * ldz + j] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      const int ntask = nig * (R >> 2);
      for (int t = threadIdx.x; t < ntask; t += blockDim.x) {
        const int rg = t / nig, ig = t - rg * nig;
        float2 acc[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int p = 0; p < 4; ++p) acc[q][p] = make_float2(0.f, 0.f);
        const float2* v0p = sV + (4 * rg) * nzp;
        const float* hp = sH + 4 * ig;
        for (int j = 0; j < nz; ++j) {
          const float4 h = *reinterpret_cast<const float4*>(hp + j * z4);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 v = v0p[q * nzp + j];
            acc[q][0].x = fmaf(h.x, v.x, acc[q][0].x);
            acc[q][0].y = fmaf(h.x, v.y, acc[q][0].y);
            acc[q][1].x = fmaf(h.y, v.x, acc[q][1].x);
            acc[q][1].y = fmaf(h.y, v.y, acc[q][1].y);
            acc[q][2].x = fmaf(h.z, v.x, acc[q][2].x);
            acc[q][2].y = fmaf(h.z, v.y, acc[q][2].y);
            acc[q][3].x = fmaf(h.w, v.x, acc[q][3].x);
            acc[q][3].y = fmaf(h.w, v.y, acc[q][3].y);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = 4 * rg + q, f = member(q);  // r & 3 == q
          if (f < 0) continue;
          float2* xo = x + (v0 + (r >> 2)) * vstride + (size_t)f * ldz;
#pragma unroll
          for (int p = 0; p < 4; ++p)
            if (4 * ig + p < nz) xo[4 * ig + p] = acc[q][p];
        }
      }
      __syncthreads();
    }
  }
}

template <int MODE>
ctof_status launch(const ctof_kernel_s* k, int nvol, const float2* vin, int ld_in, size_t in_vstride, float2* vout,
                   int ld_out, size_t out_vstride, const float* hinv, cudaStream_t st) {
  if (nvol < 1) return CTOF_EINVAL;
  // Many volumes per class: one W stage and a deep vector ring (the block is
  // reused nvol times, and the smaller footprint lets two CTAs share an SM).
  // Few volumes: whichever of (two W stages, deepest vector pipeline that fits)
  // and (one W stage, vectors one step ahead) puts more CTAs on an SM: the
  // phases of a class run between block-wide barriers, so another CTA's class
  // hides them better than a prefetch inside one CTA does.
  auto per_sm_of = [](size_t bytes) { return (int)((228 * 1024) / (bytes + 1024)); };
  int nbuf = 1, nvs = 1;
  if (nvol >= 4 && make_plan(MODE, k->nt, k->nz, 1, 4, CT_THREADS).total <= SMEM_LIMIT) {
    nvs = 4;
  } else {
    for (int v = (nvol + 1 < 4 ? nvol + 1 : 4); v >= 2; --v) {
      if (make_plan(MODE, k->nt, k->nz, 2, v, CT_THREADS).total <= SMEM_LIMIT) {
        nbuf = 2;
        nvs = v;
        break;
      }
    }
    const size_t one = make_plan(MODE, k->nt, k->nz, 1, 2, CT_THREADS).total;
    const size_t cur = make_plan(MODE, k->nt, k->nz, nbuf, nvs, CT_THREADS).total;
    if (one <= SMEM_LIMIT && per_sm_of(one) > per_sm_of(cur)) {
      nbuf = 1;
      nvs = 2;
    }
  }
  const Plan p = make_plan(MODE, k->nt, k->nz, nbuf, nvs, CT_THREADS);
  if (p.total > SMEM_LIMIT) return CTOF_EUNSUPPORTED;
  CTOF_CUDA_TRY(cudaFuncSetAttribute(k_contract<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.total));
  int per_sm = (int)((228 * 1024) / (p.total + 1024 + 64));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 4) per_sm = 4;
  int grid = 152 * per_sm;
  if (grid > k->nclass) grid = k->nclass;
  k_contract<MODE><<<grid, CT_THREADS, p.total, st>>>(k->d_what, k->d_members, k->nclass, k->nt, k->nz, vin, ld_in,
                                                      in_vstride, vout, ld_out, out_vstride, nvol, hinv, nbuf, nvs);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

}  // namespace

size_t contract_smem_bytes(int nt, int nz) {
  size_t worst = 0;
  for (int mode = MODE_FWD; mode <= MODE_TIK; ++mode) {
    const size_t b = make_plan(mode, nt, nz, 1, 1, CT_THREADS).total;
    worst = b > worst ? b : worst;
  }
  return worst;
}

ctof_status contract_forward(const ctof_kernel_s* k, const float2* in_z, float2* out_t, cudaStream_t st) {
  return contract_forward_batch(k, 1, in_z, out_t, st);
}

ctof_status contract_adjoint(const ctof_kernel_s* k, const float2* in_t, float2* out_z, cudaStream_t st) {
  return contract_adjoint_batch(k, 1, in_t, out_z, st);
}

ctof_status contract_tikhonov(const ctof_kernel_s* k, const float* hinv, const float2* m_hat, float2* x_hat,
                              cudaStream_t st) {
  return contract_tikhonov_batch(k, 1, hinv, m_hat, x_hat, st);
}

// From this many volumes on, the batched forward and adjoint run as one
// 128-wide tensor-core GEMM per frequency class (contract_tc.cu); below it the
// per-volume FP32 path above streams the class block once for all volumes.
constexpr int TC_MIN_VOLUMES = 4;

ctof_status contract_forward_batch(const ctof_kernel_s* k, int nvol, const float2* in_z, float2* out_t,
                                   cudaStream_t st) {
  if (nvol >= TC_MIN_VOLUMES) return contract_tc_forward(k, nvol, in_z, out_t, st);
  return launch<MODE_FWD>(k, nvol, in_z, k->ldz, (size_t)k->nf * k->ldz, out_t, k->ldt, (size_t)k->nf * k->ldt,
                          nullptr, st);
}

ctof_status contract_adjoint_batch(const ctof_kernel_s* k, int nvol, const float2* in_t, float2* out_z,
                                   cudaStream_t st) {
  if (nvol >= TC_MIN_VOLUMES) return contract_tc_adjoint(k, nvol, in_t, out_z, st);
  return launch<MODE_ADJ>(k, nvol, in_t, k->ldt, (size_t)k->nf * k->ldt, out_z, k->ldz, (size_t)k->nf * k->ldz,
                          nullptr, st);
}

namespace {

// x[v][f][:] <- Hinv_c x[v][f][:] for every class member f and volume v; volume v
// of frequency f at x + v * vstride + f * ld.
ctof_status apply_hinv(const ctof_kernel_s* k, int nvol, const float* hinv, float2* x, int ld, size_t vstride,
                       cudaStream_t st) {
  const int z4 = (k->nz + 3) & ~3;
  const size_t sm = (size_t)k->nz * z4 * 4 + (size_t)HV * 4 * (k->nz + 1) * 8;
  CTOF_CUDA_TRY(cudaFuncSetAttribute(k_apply_hinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, k->device);
  const int per_sm = (int)((228 * 1024) / (sm + 1024)) < 4 ? (int)((228 * 1024) / (sm + 1024)) : 4;
  const int grid = k->nclass < per_sm * nsm ? k->nclass : per_sm * nsm;
  k_apply_hinv<<<grid, 256, sm, st>>>(hinv, k->d_members, k->nclass, k->nz, z4, nvol, x, ld, vstride);
  CTOF_CUDA_TRY(cudaGetLastError());
  return CTOF_OK;
}

}  // namespace

ctof_status contract_tikhonov_zb(const ctof_kernel_s* k, int nvol, const float* hinv, const float2* m_hat,
                                 float2* x_hat, int ldzb, cudaStream_t st) {
  CTOF_TRY(contract_tc_adjoint_zb(k, nvol, m_hat, x_hat, ldzb, st));
  return apply_hinv(k, nvol, hinv, x_hat, ldzb, (size_t)k->nz, st);
}

ctof_status contract_tikhonov_batch(const ctof_kernel_s* k, int nvol, const float* hinv, const float2* m_hat,
                                    float2* x_hat, cudaStream_t st) {
  if (nvol >= TC_MIN_VOLUMES) {
    // W_hat^T m_hat on the tensor cores, then the per-class inverse in place
    CTOF_TRY(contract_tc_adjoint(k, nvol, m_hat, x_hat, st));
    return apply_hinv(k, nvol, hinv, x_hat, k->ldz, (size_t)k->nf * k->ldz, st);
  }
  return launch<MODE_TIK>(k, nvol, m_hat, k->ldt, (size_t)k->nf * k->ldt, x_hat, k->ldz, (size_t)k->nf * k->ldz, hinv,
                          st);
}
