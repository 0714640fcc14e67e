// C ABI entry points: argument validation, the handle and its workspaces, and
// the orchestration of the forward / adjoint / reconstruction chains.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "ctof_internal.h"

static thread_local char g_last_error[512] = "";

void ctof_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s (%s) at %s:%d: %s", cudaGetErrorName(e), what, file, line,
           cudaGetErrorString(e));
}

void ctof_set_last_error_text(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

namespace {


bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

ctof_status validate(const ctof_optics* o, const ctof_grid* g) {
  if (!o || !g) return CTOF_EINVAL;
  if (!(isfinite(o->mua_mm) && o->mua_mm >= 0.0) || !finite_pos(o->musp_mm) || !(isfinite(o->n) && o->n >= 1.0))
    return CTOF_EINVAL;
  if (!isfinite(o->z0_mm)) return CTOF_EINVAL;
  if (g->nx <= 0 || g->ny <= 0 || g->nz <= 0 || g->nt <= 0) return CTOF_EINVAL;
  if (!finite_pos(g->dx_mm) || !finite_pos(g->dy_mm) || !finite_pos(g->dz_mm) || !finite_pos(g->z_first_mm) ||
      !finite_pos(g->dt_ps))
    return CTOF_EINVAL;
  if (g->conv_mode != CTOF_LINEAR && g->conv_mode != CTOF_CIRCULAR) return CTOF_EINVAL;
  if (g->nx != g->ny) return CTOF_EUNSUPPORTED;
  if (g->nz > 64 || g->nt > 1024) return CTOF_EUNSUPPORTED;
  // one frequency class (W_hat block, vectors, partial sums) must fit in shared memory
  {
    const size_t admm = contract_admm_smem_bytes(g->nt, g->nz, 1);
    const size_t other = contract_smem_bytes(g->nt, g->nz);
    if (admm > 227 * 1024 || other > 227 * 1024) return CTOF_EUNSUPPORTED;
  }
  if (g->conv_mode == CTOF_LINEAR) {
    if (g->nx < 4 || g->nx > 256) return CTOF_EUNSUPPORTED;
  } else {
    if (g->nx < 32 || g->nx > 512 || (g->nx & (g->nx - 1)) != 0) return CTOF_EUNSUPPORTED;
  }
  return CTOF_OK;
}

// Frequency classes: half-plane frequencies with equal W_hat.  The kernel is
// even in x and y (and symmetric under x <-> y when dx == dy), so W_hat(kx,ky)
// depends on (kx, |ky|) -- and on the unordered pair when symmetric.
void make_classes(int P, bool symmetric, std::vector<int>& members, std::vector<float>& lap) {
  const int h = P / 2 + 1;
  const int A = h;
  std::vector<int> key_to_class((size_t)A * A, -1);
  std::vector<std::pair<int, int>> keys;
  // enumerate keys in (b, a) order so that class 0 is the DC frequency
  for (int b = 0; b < A; ++b)
    for (int a = 0; a < A; ++a) {
      if (symmetric && a > b) continue;
      key_to_class[(size_t)b * A + a] = (int)keys.size();
      keys.push_back({a, b});
    }
  const int nclass = (int)keys.size();
  members.assign((size_t)nclass * 4, -1);
  std::vector<int> count(nclass, 0);
  for (int ky = 0; ky < P; ++ky)
    for (int kx = 0; kx < h; ++kx) {
      int a = kx, b = ky <= P / 2 ? ky : P - ky;
      if (symmetric && a > b) std::swap(a, b);
      const int c = key_to_class[(size_t)b * A + a];
      const int f = ky * h + kx;
      members[(size_t)c * 4 + count[c]++] = f;
    }
  // the class's first member must be (kx = a, |ky| = b) for the table gather
  for (int c = 0; c < nclass; ++c) {
    const int a = keys[c].first, b = keys[c].second;
    for (int m = 0; m < count[c]; ++m) {
      const int f = members[(size_t)c * 4 + m];
      const int kx = f % h, ky = f / h;
      if (kx == a && (ky == b || ky == (P - b) % P)) {
        std::swap(members[(size_t)c * 4], members[(size_t)c * 4 + m]);
        break;
      }
    }
  }
  lap.resize(nclass);
  const double pi = 3.14159265358979323846;
  for (int c = 0; c < nclass; ++c) {
    const double sa = sin(pi * keys[c].first / P), sb = sin(pi * keys[c].second / P);
    lap[c] = (float)(4.0 * sa * sa + 4.0 * sb * sb);
  }
}

struct Carver {
  size_t off = 0;
  template <typename T>
  size_t take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    const size_t at = off;
    off += count * sizeof(T);
    return at;
  }
};

ctof_status forward_impl(ctof_kernel_s* k, const float* mu, float* m, cudaStream_t st) {
  CTOF_TRY(fft_forward_planes(k, mu, k->nz, k->n, k->n, k->n, k->d_inter_z, k->d_spec_z, k->ldz, st));
  CTOF_TRY(contract_forward(k, k->d_spec_z, k->d_spec_t, st));
  return fft_inverse_planes(k, k->d_spec_t, k->ldt, k->nt, k->n, k->n, k->d_inter_t, m, k->n, st);
}

ctof_status adjoint_impl(ctof_kernel_s* k, const float* m, float* vol, cudaStream_t st) {
  CTOF_TRY(fft_forward_planes(k, m, k->nt, k->n, k->n, k->n, k->d_inter_t, k->d_spec_t, k->ldt, st));
  CTOF_TRY(contract_adjoint(k, k->d_spec_t, k->d_spec_z, st));
  return fft_inverse_planes(k, k->d_spec_z, k->ldz, k->nz, k->n, k->n, k->d_inter_z, vol, k->n, st);
}

// ADMM set-up on the staged measurement d_mstage: the TV weight and the state reset.
ctof_status admm_setup(ctof_kernel_s* k, const ctof_solver_params* prm, cudaStream_t st) {
  const int nt = k->nt, nz = k->nz, n = k->n, P = k->p;
  const size_t pp = (size_t)P * P;
  CTOF_CUDA_TRY(cudaMemsetAsync(k->d_scalars, 0, 16 * sizeof(double), st));
  if (prm->tv_beta < 0) {
    CTOF_TRY(adjoint_impl(k, k->d_mstage, k->d_vstage, st));
    CTOF_TRY(reduce_max_abs(k->d_vstage, (size_t)nz * n * n, k->d_scalars + 1, st));
  }
  CTOF_TRY(admm_set_beta(k->d_scalars, prm->tv_beta, prm->beta_rel, 1.0 / (k->scale * k->scale), st));
  CTOF_CUDA_TRY(cudaMemsetAsync(k->d_spec_t2, 0, (size_t)k->nf * k->ldt * sizeof(float2), st));
  CTOF_CUDA_TRY(cudaMemsetAsync(k->d_spec_z, 0, (size_t)k->nf * k->ldz * sizeof(float2), st));
  CTOF_CUDA_TRY(cudaMemsetAsync(k->d_spec_z2, 0, (size_t)k->nf * k->ldz * sizeof(float2), st));
  CTOF_CUDA_TRY(cudaMemsetAsync(k->d_u1, 0, (size_t)nt * n * n * sizeof(float), st));
  CTOF_CUDA_TRY(cudaMemsetAsync(k->d_u2a, 0, 3 * nz * pp * sizeof(float), st));
  CTOF_CUDA_TRY(cudaMemsetAsync(k->d_u3, 0, nz * pp * sizeof(float), st));
  return CTOF_OK;
}

// The x-update of iteration `it` (per frequency class) and K x.
ctof_status admm_contract(ctof_kernel_s* k, cudaStream_t st) {
  return contract_admm(k, k->d_spec_t2, k->d_spec_z, k->d_spec_z2, k->d_spec_t, (float)(1.0 / k->scale), st);
}

// The rest of iteration `it`: T side (K x -> v1/u1 -> c_hat; not after the
// last iteration) and Z side (x -> TV / nonnegativity prox -> s_hat; the last
// iteration writes the crop of v3 to d_vstage).  `ev_mid` (optional) is
// recorded between the two.
ctof_status admm_side(ctof_kernel_s* k, const ctof_solver_params* prm, int it, cudaStream_t st, cudaEvent_t ev_mid) {
  const int nt = k->nt, nz = k->nz, n = k->n, P = k->p;
  const float inv_s = (float)(1.0 / k->scale);
  const float rho = (float)prm->rho;
  const bool last = it == prm->iters - 1;
  if (!last) {
    CTOF_TRY(fft_cols_inverse(k, k->d_spec_t, k->ldt, nt, n, k->d_inter_t, st));
    CTOF_TRY(fft_rows_admm_t(k, k->d_inter_t, k->d_mstage, k->d_u1, inv_s, rho, st));
    CTOF_TRY(fft_cols_forward(k, k->d_inter_t, nt, n, k->d_spec_t2, k->ldt, st));
  }
  if (ev_mid) CTOF_CUDA_TRY(cudaEventRecordWithFlags(ev_mid, st, cudaEventRecordExternal));
  float* u2[2] = {k->d_u2a, k->d_u2b};
  CTOF_TRY(fft_cols_inverse(k, k->d_spec_z2, k->ldz, nz, P, k->d_inter_z, st));
  CTOF_TRY(fft_rows_inverse(k, k->d_inter_z, nz, P, P, k->d_xs, P, st));
  CTOF_TRY(admm_tv_stencil(k, k->d_xs, u2[it & 1], u2[(it + 1) & 1], k->d_u3, k->d_s, k->d_scalars, rho,
                           last ? k->d_vstage : nullptr, st));
  if (!last) {
    CTOF_TRY(fft_rows_forward(k, k->d_s, nz, P, P, P, k->d_inter_z, st));
    CTOF_TRY(fft_cols_forward(k, k->d_inter_z, nz, P, k->d_spec_z, k->ldz, st));
  }
  return CTOF_OK;
}

// ADMM on the staged measurement d_mstage; result (crop of v3) in d_vstage.
ctof_status admm_enqueue(ctof_kernel_s* k, const ctof_solver_params* prm, cudaStream_t st, bool timed) {
  CTOF_TRY(admm_setup(k, prm, st));
  cudaEvent_t* ev = (timed && k->timing) ? k->events : nullptr;
  for (int it = 0; it < prm->iters; ++it) {
    if (ev) CTOF_CUDA_TRY(cudaEventRecordWithFlags(ev[4 * it + 0], st, cudaEventRecordExternal));
    CTOF_TRY(admm_contract(k, st));
    if (ev) CTOF_CUDA_TRY(cudaEventRecordWithFlags(ev[4 * it + 1], st, cudaEventRecordExternal));
    CTOF_TRY(admm_side(k, prm, it, st, ev ? ev[4 * it + 2] : nullptr));
    if (ev) CTOF_CUDA_TRY(cudaEventRecordWithFlags(ev[4 * it + 3], st, cudaEventRecordExternal));
  }
  return CTOF_OK;
}

void destroy_events(ctof_kernel_s* k) {
  for (int i = 0; i < k->n_events; ++i) cudaEventDestroy(k->events[i]);
  delete[] k->events;
  k->events = nullptr;
  k->n_events = 0;
}

ctof_status ensure_events(ctof_kernel_s* k, int count) {
  if (k->n_events >= count) return CTOF_OK;
  destroy_events(k);
  k->events = new (std::nothrow) cudaEvent_t[count];
  if (!k->events) return CTOF_ENOMEM;
  for (int i = 0; i < count; ++i) {
    if (cudaEventCreate(&k->events[i]) != cudaSuccess) {
      k->n_events = i;
      destroy_events(k);
      return CTOF_ECUDA;
    }
  }
  k->n_events = count;
  return CTOF_OK;
}

// Autotuner: times each column-pass tile (32 columns of 8 or 16 planes, 16
// columns of 8 or 16 planes) on the handle's own buffers for the four
// column-pass shapes of an ADMM iteration and keeps the fastest.
// Synchronous; must run outside stream capture.
ctof_status autotune(ctof_kernel_s* k, cudaStream_t st) {
  if (k->tuned) return CTOF_OK;
  // tile codes: 8 / 16 planes in 32-column tiles, 100 + 8 / 16 in 16-column tiles
  const int cands[4] = {8, 16, 108, 116};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CTOF_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return CTOF_ECUDA;
  }
  ctof_status s = CTOF_OK;
  const int n = k->n, P = k->p;
  if (cudaMemsetAsync(k->d_inter_t, 0, fft_inter_elems(k, k->nt, n) * sizeof(float2), st) != cudaSuccess ||
      cudaMemsetAsync(k->d_inter_z, 0, fft_inter_elems(k, k->nz, P) * sizeof(float2), st) != cudaSuccess ||
      cudaMemsetAsync(k->d_spec_t, 0, (size_t)k->nf * k->ldt * sizeof(float2), st) != cudaSuccess ||
      cudaMemsetAsync(k->d_spec_z2, 0, (size_t)k->nf * k->ldz * sizeof(float2), st) != cudaSuccess)
    s = CTOF_ECUDA;
  for (int use = 0; use < 4 && s == CTOF_OK; ++use) {
    float best_ms = 1e30f;
    int best = 16;
    for (int ci = 0; ci < 4 && s == CTOF_OK; ++ci) {
      const int pb = cands[ci];
      auto launch = [&]() -> ctof_status {
        switch (use) {
          case 0: return fft_cols_forward_pb(k, k->d_inter_t, k->nt, n, k->d_spec_t2, k->ldt, pb, st);
          case 1: return fft_cols_inverse_pb(k, k->d_spec_t, k->ldt, k->nt, n, k->d_inter_t, pb, st);
          case 2: return fft_cols_forward_pb(k, k->d_inter_z, k->nz, P, k->d_spec_z, k->ldz, pb, st);
          default: return fft_cols_inverse_pb(k, k->d_spec_z2, k->ldz, k->nz, P, k->d_inter_z, pb, st);
        }
      };
      s = launch();
      if (s != CTOF_OK) break;
      if (cudaEventRecord(e0, st) != cudaSuccess) { s = CTOF_ECUDA; break; }
      for (int r = 0; r < 3 && s == CTOF_OK; ++r) s = launch();
      if (s != CTOF_OK) break;
      float ms = 0.f;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        s = CTOF_ECUDA;
        break;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = pb;
      }
    }
    k->tune_pb[use] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s == CTOF_OK) k->tuned = 1;
  return s;
}

ctof_status admm_run(ctof_kernel_s* k, const ctof_solver_params* prm, cudaStream_t st) {
  CTOF_TRY(autotune(k, st));
  const bool same = k->graph && k->graph_iters == prm->iters && k->graph_rho == prm->rho &&
                    k->graph_beta == prm->tv_beta && k->graph_beta_rel == prm->beta_rel &&
                    k->graph_timing == k->timing;
  if (!same) {
    if (k->graph) {
      cudaGraphExecDestroy(k->graph);
      k->graph = nullptr;
    }
    if (k->timing) CTOF_TRY(ensure_events(k, 4 * prm->iters));
    cudaStream_t cap = nullptr;
    CTOF_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cap);
      CTOF_CUDA_TRY(e);
    }
    const ctof_status s = admm_enqueue(k, prm, cap, true);
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (s != CTOF_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    CTOF_CUDA_TRY(e);
    {
      size_t nn = 0;
      int kernels = 0;
      if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
          for (size_t i = 0; i < nn; ++i) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
          }
      }
      k->graph_kernel_nodes = kernels;
    }
    e = cudaGraphInstantiate(&k->graph, g, 0);
    cudaGraphDestroy(g);
    CTOF_CUDA_TRY(e);
    k->graph_timing = k->timing;
    k->graph_iters = prm->iters;
    k->graph_rho = prm->rho;
    k->graph_beta = prm->tv_beta;
    k->graph_beta_rel = prm->beta_rel;
  }
  CTOF_CUDA_TRY(cudaGraphLaunch(k->graph, st));
  return CTOF_OK;
}

}  // namespace

ctof_status tikhonov_inverse(ctof_kernel_s* k, double lambda, const float** hinv, cudaStream_t st) {
  if (!(lambda > 0.0) || !isfinite(lambda)) return CTOF_EINVAL;
  int slot = k->tik_lambda[0] == lambda ? 0 : (k->tik_lambda[1] == lambda ? 1 : -1);
  if (slot < 0) {
    slot = 1 - k->tik_last;  // replace the slot not used last
    if (!k->d_tik_hinv[slot]) {
      void* p = nullptr;
      if (cudaMalloc(&p, (size_t)k->nclass * k->nz * k->z4 * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return CTOF_ENOMEM;
      }
      k->d_tik_hinv[slot] = static_cast<float*>(p);
    }
    k->tik_lambda[slot] = -1.0;
    CTOF_TRY(build_tikhonov_factors(k, slot, lambda, st));
  }
  k->tik_last = slot;
  *hinv = k->d_tik_hinv[slot];
  return CTOF_OK;
}

namespace {

ctof_status tikhonov_run(ctof_kernel_s* k, const ctof_solver_params* prm, cudaStream_t st, double* lambda_out) {
  const double lambda = prm->tik_lambda_rel * k->gram_max;
  const float* hinv = nullptr;
  CTOF_TRY(tikhonov_inverse(k, lambda, &hinv, st));
  *lambda_out = lambda;
  CTOF_CUDA_TRY(cudaMemsetAsync(k->d_scalars, 0, 16 * sizeof(double), st));
  CTOF_TRY(fft_forward_planes(k, k->d_mstage, k->nt, k->n, k->n, k->n, k->d_inter_t, k->d_spec_t, k->ldt, st));
  CTOF_TRY(contract_tikhonov(k, hinv, k->d_spec_t, k->d_spec_z, st));
  return fft_inverse_planes(k, k->d_spec_z, k->ldz, k->nz, k->n, k->n, k->d_inter_z, k->d_vstage, k->n, st);
}

// FISTA for Eq. 10 on the staged measurement (result in d_vstage).  Normalised
// units (A_n = A / s, step 1); lam0 by the same rule as the ADMM TV weight;
// lam(z) follows the DC depth sensitivity.  With `mux` the operator is the
// composite S A of Eq. 12 (S = H_64 on every 8 x 8 block of scan points, so
// the normalisation is 8 s) and the staged measurement is the multiplexed y.
// Workspace: ADMM state buffers.
ctof_status fista_run(ctof_kernel_s* k, const ctof_solver_params* prm, bool mux, cudaStream_t st) {
  const size_t vol = (size_t)k->nz * k->n * k->n, meas = (size_t)k->nt * k->n * k->n;
  float* y = k->d_u3;
  float* x = k->d_xs;
  float* g = k->d_s;
  float* r = k->d_u1;
  float* lam = k->d_u2a;
  const double sc = k->scale * (mux ? 8.0 : 1.0);
  const float inv_s2 = (float)(1.0 / (sc * sc));
  CTOF_CUDA_TRY(cudaMemsetAsync(k->d_scalars, 0, 16 * sizeof(double), st));
  if (prm->tv_beta < 0) {
    if (mux) {
      CTOF_CUDA_TRY(cudaMemcpyAsync(r, k->d_mstage, meas * sizeof(float), cudaMemcpyDeviceToDevice, st));
      CTOF_TRY(block_hadamard(r, k->nt, k->n, st));
      CTOF_TRY(adjoint_impl(k, r, k->d_vstage, st));
    } else {
      CTOF_TRY(adjoint_impl(k, k->d_mstage, k->d_vstage, st));
    }
    CTOF_TRY(reduce_max_abs(k->d_vstage, vol, k->d_scalars + 1, st));
  }
  CTOF_TRY(admm_set_beta(k->d_scalars, prm->tv_beta, prm->beta_rel, 1.0 / (sc * sc), st));
  CTOF_TRY(fista_lambda(k, k->d_scalars, lam, st));
  CTOF_CUDA_TRY(cudaMemsetAsync(y, 0, vol * sizeof(float), st));
  CTOF_CUDA_TRY(cudaMemsetAsync(x, 0, vol * sizeof(float), st));
  double t = 1.0;
  for (int it = 0; it < prm->iters; ++it) {
    CTOF_TRY(forward_impl(k, y, r, st));
    if (mux) CTOF_TRY(block_hadamard(r, k->nt, k->n, st));
    CTOF_TRY(fista_sub_meas(r, k->d_mstage, meas, st));
    if (mux) CTOF_TRY(block_hadamard(r, k->nt, k->n, st));  // S^T = S
    CTOF_TRY(adjoint_impl(k, r, g, st));
    const double t_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    CTOF_TRY(fista_step(y, g, x, lam, (float)((t - 1.0) / t_next), inv_s2, k->n * k->n, vol, st));
    t = t_next;
  }
  CTOF_CUDA_TRY(cudaMemcpyAsync(k->d_vstage, x, vol * sizeof(float), cudaMemcpyDeviceToDevice, st));
  return CTOF_OK;
}

ctof_status validate_params(const ctof_solver_params* p) {
  if (!p) return CTOF_EINVAL;
  if (p->solver == CTOF_SOLVER_FISTA_L1 || p->solver == CTOF_SOLVER_FISTA_L1_MUX) {
    if (p->iters < 1 || p->iters > 100000) return CTOF_EINVAL;
    if (!isfinite(p->tv_beta)) return CTOF_EINVAL;
    if (p->tv_beta < 0 && !(isfinite(p->beta_rel) && p->beta_rel >= 0)) return CTOF_EINVAL;
    return CTOF_OK;
  }
  if (p->solver == CTOF_SOLVER_ADMM_TV) {
    if (p->iters < 1 || p->iters > 100000) return CTOF_EINVAL;
    if (!finite_pos(p->rho)) return CTOF_EINVAL;
    if (!isfinite(p->tv_beta)) return CTOF_EINVAL;
    if (p->tv_beta < 0 && !(isfinite(p->beta_rel) && p->beta_rel >= 0)) return CTOF_EINVAL;
    return CTOF_OK;
  }
  if (p->solver == CTOF_SOLVER_TIKHONOV) return finite_pos(p->tik_lambda_rel) ? CTOF_OK : CTOF_EINVAL;
  return CTOF_EINVAL;
}

// Runs the chosen solver on d_mstage, leaving the result in d_vstage.
ctof_status solve_staged(ctof_kernel_s* k, const ctof_solver_params* prm, double* lambda, cudaStream_t st) {
  *lambda = 0.0;
  if (prm->solver == CTOF_SOLVER_ADMM_TV) return admm_run(k, prm, st);
  if (prm->solver == CTOF_SOLVER_FISTA_L1) return fista_run(k, prm, false, st);
  if (prm->solver == CTOF_SOLVER_FISTA_L1_MUX) {
    if (k->n % 8 != 0) return CTOF_EUNSUPPORTED;
    return fista_run(k, prm, true, st);
  }
  return tikhonov_run(k, prm, st, lambda);
}

}  // namespace

ctof_status take_device_status(ctof_kernel_s* k, cudaStream_t st) {
  int flag = 0;
  CTOF_CUDA_TRY(cudaMemcpyAsync(&flag, k->d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  CTOF_CUDA_TRY(cudaMemsetAsync(k->d_flags, 0, sizeof(int), st));
  CTOF_CUDA_TRY(cudaStreamSynchronize(st));
  return flag ? CTOF_ETIMEOUT : CTOF_OK;
}

namespace {

// Synchronising report: parameters used, a NaN/Inf scan of the result, and
// the handle's sticky device status (a bounded wait that ran out).
ctof_status fill_report(ctof_kernel_s* k, const ctof_solver_params* prm, double lambda, ctof_report* rep,
                        cudaStream_t st) {
  int* flag = reinterpret_cast<int*>(k->d_scalars + 8);
  CTOF_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
  CTOF_TRY(check_finite(k->d_vstage, (size_t)k->nz * k->n * k->n, flag, st));
  double sc[10];
  CTOF_CUDA_TRY(cudaMemcpyAsync(sc, k->d_scalars, 10 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CTOF_CUDA_TRY(cudaStreamSynchronize(st));
  int bad = 0;
  memcpy(&bad, &sc[8], sizeof(int));
  const ctof_status waits = take_device_status(k, st);
  rep->scale = k->scale;
  rep->beta = prm->solver == CTOF_SOLVER_TIKHONOV ? 0.0 : sc[0];
  rep->lambda = lambda;
  rep->iters_done = prm->solver == CTOF_SOLVER_TIKHONOV ? 1 : prm->iters;
  if (waits != CTOF_OK) return waits;
  return bad ? CTOF_ENONFINITE : CTOF_OK;
}

// One graph per distinct batch (handles, buffers, parameters): every problem's
// ADMM chain is captured on its own forked stream so that the problems run
// concurrently on the GPU; the graph is replayed while the batch repeats.
struct BatchGraph {
  std::vector<unsigned long long> uids;
  std::vector<const void*> ptrs;
  int iters = 0;
  double rho = 0, beta = 0, beta_rel = 0;
  cudaGraphExec_t exec = nullptr;
  AdmmQueue queue;  // the batched x-update's problem table and work-queue counter
};
std::mutex g_batch_mutex;
BatchGraph g_batch;
std::vector<cudaStream_t> g_side_streams;
std::vector<cudaEvent_t> g_side_events;

ctof_status batch_graph_run(int count, const ctof_kernel* ks, const float* const* d_m,
                            const ctof_solver_params* prm, float* const* d_mu, cudaStream_t st) {
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  std::vector<unsigned long long> uids(count);
  std::vector<const void*> ptrs(2 * count);
  for (int i = 0; i < count; ++i) {
    uids[i] = ks[i]->uid;
    ptrs[2 * i] = d_m[i];
    ptrs[2 * i + 1] = d_mu[i];
  }
  const bool same = g_batch.exec && g_batch.uids == uids && g_batch.ptrs == ptrs && g_batch.iters == prm->iters &&
                    g_batch.rho == prm->rho && g_batch.beta == prm->tv_beta && g_batch.beta_rel == prm->beta_rel;
  if (!same) {
    if (g_batch.exec) {
      cudaGraphExecDestroy(g_batch.exec);
      g_batch.exec = nullptr;
    }
    const int nside = count < 32 ? count : 32;
    while ((int)g_side_streams.size() < nside) {
      cudaStream_t s2 = nullptr;
      CTOF_CUDA_TRY(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
      g_side_streams.push_back(s2);
    }
    while ((int)g_side_events.size() < nside + 1) {
      cudaEvent_t e = nullptr;
      CTOF_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      g_side_events.push_back(e);
    }
    // problems whose x-update runs in the one persistent queue launch per iteration
    CTOF_TRY(admm_queue_build(count, const_cast<ctof_kernel_s* const*>(ks), &g_batch.queue));
    std::vector<char> queued(count, 0);
    for (int i : g_batch.queue.members) queued[i] = 1;
    cudaStream_t cap = nullptr;
    CTOF_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    ctof_status s = e == cudaSuccess ? CTOF_OK : CTOF_ECUDA;
    // fork the side streams off `cap`, or join them back into it
    auto fork = [&]() {
      if (s == CTOF_OK && cudaEventRecord(g_side_events[nside], cap) != cudaSuccess) s = CTOF_ECUDA;
      for (int j = 0; j < nside && s == CTOF_OK; ++j)
        if (cudaStreamWaitEvent(g_side_streams[j], g_side_events[nside], 0) != cudaSuccess) s = CTOF_ECUDA;
    };
    auto join = [&]() {
      for (int j = 0; j < nside && s == CTOF_OK; ++j) {
        if (cudaEventRecord(g_side_events[j], g_side_streams[j]) != cudaSuccess ||
            cudaStreamWaitEvent(cap, g_side_events[j], 0) != cudaSuccess)
          s = CTOF_ECUDA;
      }
    };
    // side streams: the problems with their own x-update launch get streams of
    // their own (they run beside the queue launch), the queued ones share the rest
    std::vector<int> stream_of(count);
    {
      int nown = 0;
      for (int i = 0; i < count; ++i) nown += !queued[i];
      const int own_streams = nown < nside / 2 ? nown : nside / 2;
      int a = 0, b = 0;
      for (int i = 0; i < count; ++i) {
        if (!queued[i] && own_streams > 0)
          stream_of[i] = (a++) % own_streams;
        else
          stream_of[i] = own_streams + (b++) % (nside - own_streams > 0 ? nside - own_streams : 1);
        if (stream_of[i] >= nside) stream_of[i] = nside - 1;
      }
    }
    fork();
    for (int i = 0; i < count && s == CTOF_OK; ++i) {
      ctof_kernel_s* k = ks[i];
      cudaStream_t side = g_side_streams[stream_of[i]];
      const size_t mb = (size_t)k->nt * k->n * k->n * sizeof(float);
      if (cudaMemcpyAsync(k->d_mstage, d_m[i], mb, cudaMemcpyDeviceToDevice, side) != cudaSuccess) s = CTOF_ECUDA;
      if (s == CTOF_OK) s = admm_setup(k, prm, side);
    }
    join();
    // iterations in lockstep: the problems with their own x-update run it and their
    // T / Z sides from the iteration's start; beside them the queued x-updates of
    // all other problems run as one launch, after which their T / Z sides follow
    cudaEvent_t ev_q = g_side_events[nside];
    for (int it = 0; it < prm->iters && s == CTOF_OK; ++it) {
      fork();
      for (int i = 0; i < count && s == CTOF_OK; ++i) {
        if (queued[i]) continue;
        cudaStream_t side = g_side_streams[stream_of[i]];
        s = admm_contract(ks[i], side);
        if (s == CTOF_OK) s = admm_side(ks[i], prm, it, side, nullptr);
      }
      if (s == CTOF_OK) s = admm_queue_launch(g_batch.queue, cap);
      if (s == CTOF_OK && cudaEventRecord(ev_q, cap) != cudaSuccess) s = CTOF_ECUDA;
      for (int i = 0; i < count && s == CTOF_OK; ++i) {
        if (!queued[i]) continue;
        cudaStream_t side = g_side_streams[stream_of[i]];
        if (cudaStreamWaitEvent(side, ev_q, 0) != cudaSuccess) s = CTOF_ECUDA;
        if (s == CTOF_OK) s = admm_side(ks[i], prm, it, side, nullptr);
      }
      join();
    }
    fork();
    for (int i = 0; i < count && s == CTOF_OK; ++i) {
      ctof_kernel_s* k = ks[i];
      const size_t vb = (size_t)k->nz * k->n * k->n * sizeof(float);
      if (cudaMemcpyAsync(d_mu[i], k->d_vstage, vb, cudaMemcpyDeviceToDevice, g_side_streams[stream_of[i]]) !=
          cudaSuccess)
        s = CTOF_ECUDA;
    }
    join();
    e = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (s == CTOF_OK && e != cudaSuccess) s = CTOF_ECUDA;
    if (s == CTOF_OK && cudaGraphInstantiate(&g_batch.exec, graph, 0) != cudaSuccess) {
      g_batch.exec = nullptr;
      s = CTOF_ECUDA;
    }
    if (graph) cudaGraphDestroy(graph);
    if (s != CTOF_OK) {
      cudaGetLastError();
      return s;
    }
    g_batch.uids = uids;
    g_batch.ptrs = ptrs;
    g_batch.iters = prm->iters;
    g_batch.rho = prm->rho;
    g_batch.beta = prm->tv_beta;
    g_batch.beta_rel = prm->beta_rel;
    // the handles' own single-problem graphs stay valid: they stage through the
    // same buffers and are not affected by this graph
  }
  CTOF_CUDA_TRY(cudaGraphLaunch(g_batch.exec, st));
  return CTOF_OK;
}

void batch_graph_forget(const ctof_kernel_s* k) {
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  for (unsigned long long u : g_batch.uids)
    if (u == k->uid && g_batch.exec) {
      cudaGraphExecDestroy(g_batch.exec);
      g_batch.exec = nullptr;
      g_batch.uids.clear();
      break;
    }
}

}  // namespace

extern "C" {

const char* ctof_status_string(ctof_status s) {
  switch (s) {
    case CTOF_OK: return "ok";
    case CTOF_EINVAL: return "invalid argument";
    case CTOF_ENOMEM: return "out of device memory";
    case CTOF_ECUDA: return "CUDA runtime error";
    case CTOF_ENONFINITE: return "non-finite value";
    case CTOF_ETIMEOUT: return "device wait timed out";
    case CTOF_EUNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

const char* ctof_last_error_message(void) { return g_last_error; }

void ctof_kernel_destroy(ctof_kernel k) {
  if (!k) return;
  DeviceGuard guard(k->device);
  batch_graph_forget(k);
  if (k->graph) cudaGraphExecDestroy(k->graph);
  destroy_events(k);
  if (k->d_bt_cinv) cudaFree(k->d_bt_cinv);
  if (k->d_batch) cudaFree(k->d_batch);
  for (int i = 0; i < 2; ++i)
    if (k->d_tik_hinv[i]) cudaFree(k->d_tik_hinv[i]);
  if (k->d_w) cudaFree(k->d_w);
  if (k->d_base) cudaFree(k->d_base);
  delete k;
}

namespace {

ctof_status build_any(const ctof_optics* optics, const ctof_emission* emission, const ctof_voxel_average* average,
                      const ctof_grid* grid, int flags, void* stream, ctof_kernel* out) {
  if (!out) return CTOF_EINVAL;
  *out = nullptr;
  CTOF_TRY(validate(optics, grid));
  if (emission && !(isfinite(emission->mua_mm) && emission->mua_mm >= 0.0 && finite_pos(emission->musp_mm) &&
                    isfinite(emission->tau_ps) && emission->tau_ps >= 0.0))
    return CTOF_EINVAL;
  if (average) {
    if (average->layers < 0 || average->layers > grid->nz || average->nodes < 1 || average->nodes > 8)
      return CTOF_EINVAL;
    if (average->layers > 0 && grid->z_first_mm < 0.5 * grid->dz_mm) return CTOF_EINVAL;
  }
  if (flags & ~CTOF_KEEP_W) return CTOF_EINVAL;
  int dev = 0;
  CTOF_CUDA_TRY(cudaGetDevice(&dev));
  ctof_kernel_s* k = new (std::nothrow) ctof_kernel_s();
  if (!k) return CTOF_ENOMEM;
  k->optics = *optics;
  k->grid = *grid;
  k->flags = flags;
  k->fluorescence = emission ? 1 : 0;
  if (emission) k->emission = *emission;
  k->avg.layers = average ? average->layers : 0;
  k->avg.nodes = average ? average->nodes : 1;
  k->device = dev;
  k->n = grid->nx;
  k->nt = grid->nt;
  k->nz = grid->nz;
  k->p = grid->conv_mode == CTOF_LINEAR ? std::max(32, next_pow2(2 * grid->nx)) : grid->nx;
  k->h = k->p / 2 + 1;
  k->hp = ctof_round_up(k->h, 4);
  k->nf = k->p * k->h;
  k->q = grid->conv_mode == CTOF_LINEAR ? grid->nx : k->p / 2 + 1;
  k->z4 = ctof_round_up(k->nz, 4);
  k->ldt = ctof_round_up(k->nt, 8);
  k->ldz = ctof_round_up(k->nz, 8);
  k->symmetric = grid->dx_mm == grid->dy_mm;
  k->r_min = optics->clamp_r ? 0.5 * std::min(grid->dx_mm, std::min(grid->dy_mm, grid->dz_mm)) : 0.0;
  k->tik_lambda[0] = k->tik_lambda[1] = -1.0;
  k->tik_last = 1;
  k->max_polls = CTOF_DEFAULT_MAX_POLLS;
  for (int i = 0; i < 4; ++i) k->tune_pb[i] = 16;
  {
    static std::atomic<unsigned long long> next_id{1};
    k->uid = next_id++;
  }

  std::vector<int> members;
  std::vector<float> lap;
  make_classes(k->p, k->symmetric != 0, members, lap);
  k->nclass = (int)lap.size();

  const int nt = k->nt, nz = k->nz, n = k->n, P = k->p;
  const size_t pp = (size_t)P * P;
  Carver cv;
  const size_t o_members = cv.take<int>((size_t)k->nclass * 4);
  const size_t o_lap = cv.take<float>(k->nclass);
  const size_t o_what = cv.take<float>((size_t)k->nclass * nt * k->z4);
  const size_t o_gram = cv.take<double>((size_t)k->nclass * nz * nz);
  const size_t o_hinv = cv.take<float>((size_t)k->nclass * nz * k->z4);
  const size_t wa_per = contract_admm_pipe_floats(nt, nz, 0), ha_per = contract_admm_pipe_floats(nt, nz, 1);
  const size_t o_wa = wa_per ? cv.take<float>((size_t)k->nclass * wa_per) : 0;
  const size_t o_ha = wa_per ? cv.take<float>((size_t)k->nclass * ha_per) : 0;
  const size_t o_tw = cv.take<float2>(fft_twiddle_count(P));
  const size_t o_st = cv.take<float2>((size_t)k->nf * k->ldt);
  const size_t o_st2 = cv.take<float2>((size_t)k->nf * k->ldt);
  const size_t o_sz = cv.take<float2>((size_t)k->nf * k->ldz);
  const size_t o_sz2 = cv.take<float2>((size_t)k->nf * k->ldz);
  const size_t o_it = cv.take<float2>(fft_inter_elems(k, nt, n));
  const size_t o_iz = cv.take<float2>(fft_inter_elems(k, nz, P));
  const size_t o_u1 = cv.take<float>((size_t)nt * n * n);
  const size_t o_ms = cv.take<float>((size_t)nt * n * n);
  const size_t o_u2a = cv.take<float>(3 * nz * pp);
  const size_t o_u2b = cv.take<float>(3 * nz * pp);
  const size_t o_u3 = cv.take<float>(nz * pp);
  const size_t o_xs = cv.take<float>(nz * pp);
  const size_t o_s = cv.take<float>(nz * pp);
  const size_t o_vs = cv.take<float>((size_t)nz * n * n);
  const size_t o_sc = cv.take<double>(16);
  const size_t o_fl = cv.take<int>(4);
  k->bytes = cv.off;
  if (cudaMalloc(&k->d_base, k->bytes) != cudaSuccess) {
    cudaGetLastError();
    delete k;
    return CTOF_ENOMEM;
  }
  char* b = static_cast<char*>(k->d_base);
  k->d_members = reinterpret_cast<int*>(b + o_members);
  k->d_lap = reinterpret_cast<float*>(b + o_lap);
  k->d_what = reinterpret_cast<float*>(b + o_what);
  k->d_gram = reinterpret_cast<double*>(b + o_gram);
  k->d_hinv = reinterpret_cast<float*>(b + o_hinv);
  k->d_what_admm = wa_per ? reinterpret_cast<float*>(b + o_wa) : nullptr;
  k->d_hinv_admm = wa_per ? reinterpret_cast<float*>(b + o_ha) : nullptr;
  k->d_tw = reinterpret_cast<float2*>(b + o_tw);
  k->d_spec_t = reinterpret_cast<float2*>(b + o_st);
  k->d_spec_t2 = reinterpret_cast<float2*>(b + o_st2);
  k->d_spec_z = reinterpret_cast<float2*>(b + o_sz);
  k->d_spec_z2 = reinterpret_cast<float2*>(b + o_sz2);
  k->d_inter_t = reinterpret_cast<float2*>(b + o_it);
  k->d_inter_z = reinterpret_cast<float2*>(b + o_iz);
  k->d_u1 = reinterpret_cast<float*>(b + o_u1);
  k->d_mstage = reinterpret_cast<float*>(b + o_ms);
  k->d_u2a = reinterpret_cast<float*>(b + o_u2a);
  k->d_u2b = reinterpret_cast<float*>(b + o_u2b);
  k->d_u3 = reinterpret_cast<float*>(b + o_u3);
  k->d_xs = reinterpret_cast<float*>(b + o_xs);
  k->d_s = reinterpret_cast<float*>(b + o_s);
  k->d_vstage = reinterpret_cast<float*>(b + o_vs);
  k->d_scalars = reinterpret_cast<double*>(b + o_sc);
  k->d_flags = reinterpret_cast<int*>(b + o_fl);
  if (flags & CTOF_KEEP_W) {
    void* p = nullptr;
    if (cudaMalloc(&p, (size_t)nt * nz * k->q * k->q * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      ctof_kernel_destroy(k);
      return CTOF_ENOMEM;
    }
    k->d_w = static_cast<double*>(p);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<float2> tw(fft_twiddle_count(P));
  fft_twiddle_table(P, tw.data());
  ctof_status s = CTOF_OK;
  do {
    if (cudaMemsetAsync(k->d_scalars, 0, 16 * sizeof(double), st) != cudaSuccess ||
        cudaMemsetAsync(k->d_flags, 0, 4 * sizeof(int), st) != cudaSuccess ||
        cudaMemcpyAsync(k->d_members, members.data(), members.size() * sizeof(int), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(k->d_lap, lap.data(), lap.size() * sizeof(float), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(k->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      s = CTOF_ECUDA;
      break;
    }
    s = build_kernel_tables(k, st);
  } while (0);
  if (s != CTOF_OK) {
    cudaStreamSynchronize(st);
    ctof_kernel_destroy(k);
    return s;
  }
  *out = k;
  return CTOF_OK;
}

}  // namespace

ctof_status ctof_build_kernel(const ctof_optics* optics, const ctof_grid* grid, int flags, void* stream,
                              ctof_kernel* out) {
  return build_any(optics, nullptr, nullptr, grid, flags, stream, out);
}

ctof_status ctof_build_kernel_ex(const ctof_optics* optics, const ctof_emission* emission,
                                 const ctof_voxel_average* average, const ctof_grid* grid, int flags, void* stream,
                                 ctof_kernel* out) {
  return build_any(optics, emission, average, grid, flags, stream, out);
}

ctof_status ctof_build_kernel_fluorescence(const ctof_optics* excitation, const ctof_emission* emission,
                                           const ctof_grid* grid, int flags, void* stream, ctof_kernel* out) {
  if (!emission) {
    if (out) *out = nullptr;
    return CTOF_EINVAL;
  }
  return build_any(excitation, emission, nullptr, grid, flags, stream, out);
}

ctof_status ctof_kernel_get_info(ctof_kernel k, ctof_kernel_info* info) {
  if (!k || !info) return CTOF_EINVAL;
  info->p = k->p;
  info->n_freq = k->nf;
  info->n_class = k->nclass;
  info->nt = k->nt;
  info->nz = k->nz;
  info->scale = k->scale;
  info->gram_max_diag = k->gram_max;
  info->admm_stages = k->d_what_admm ? contract_admm_pipe_stages(k->nt, k->nz) : 0;
  const size_t tik_bytes = (size_t)k->nclass * k->nz * k->z4 * sizeof(float);
  info->device_bytes = k->bytes + (k->d_w ? (size_t)k->nt * k->nz * k->q * k->q * sizeof(double) : 0) +
                       ((k->d_tik_hinv[0] ? 1 : 0) + (k->d_tik_hinv[1] ? 1 : 0)) * tik_bytes;
  return CTOF_OK;
}

ctof_status ctof_kernel_get_w(ctof_kernel k, double* h_w) {
  if (!k || !h_w) return CTOF_EINVAL;
  if (!k->d_w) return CTOF_EUNSUPPORTED;
  DeviceGuard g(k->device);
  CTOF_CUDA_TRY(cudaMemcpy(h_w, k->d_w, (size_t)k->nt * k->nz * k->q * k->q * sizeof(double), cudaMemcpyDeviceToHost));
  return CTOF_OK;
}

ctof_status ctof_kernel_get_classes(ctof_kernel k, int* h_members) {
  if (!k || !h_members) return CTOF_EINVAL;
  DeviceGuard g(k->device);
  CTOF_CUDA_TRY(cudaMemcpy(h_members, k->d_members, (size_t)k->nclass * 4 * sizeof(int), cudaMemcpyDeviceToHost));
  return CTOF_OK;
}

ctof_status ctof_kernel_get_what(ctof_kernel k, float* h_what) {
  if (!k || !h_what) return CTOF_EINVAL;
  DeviceGuard g(k->device);
  CTOF_CUDA_TRY(cudaMemcpy2D(h_what, (size_t)k->nz * sizeof(float), k->d_what, (size_t)k->z4 * sizeof(float),
                             (size_t)k->nz * sizeof(float), (size_t)k->nclass * k->nt, cudaMemcpyDeviceToHost));
  return CTOF_OK;
}

ctof_status ctof_forward(ctof_kernel k, const float* d_mu, float* d_m, void* stream) {
  if (!k || !d_mu || !d_m) return CTOF_EINVAL;
  DeviceGuard g(k->device);
  if (!g.ok) return CTOF_ECUDA;
  return forward_impl(k, d_mu, d_m, static_cast<cudaStream_t>(stream));
}

ctof_status ctof_adjoint(ctof_kernel k, const float* d_m, float* d_vol, void* stream) {
  if (!k || !d_m || !d_vol) return CTOF_EINVAL;
  DeviceGuard g(k->device);
  if (!g.ok) return CTOF_ECUDA;
  return adjoint_impl(k, d_m, d_vol, static_cast<cudaStream_t>(stream));
}

ctof_status ctof_contract_forward_batch(ctof_kernel k, int nvol, const float* d_in, float* d_out, void* stream) {
  if (!k || !d_in || !d_out || nvol < 1) return CTOF_EINVAL;
  DeviceGuard g(k->device);
  if (!g.ok) return CTOF_ECUDA;
  return contract_forward_batch(k, nvol, reinterpret_cast<const float2*>(d_in), reinterpret_cast<float2*>(d_out),
                                static_cast<cudaStream_t>(stream));
}

ctof_status ctof_contract_adjoint_batch(ctof_kernel k, int nvol, const float* d_in, float* d_out, void* stream) {
  if (!k || !d_in || !d_out || nvol < 1) return CTOF_EINVAL;
  DeviceGuard g(k->device);
  if (!g.ok) return CTOF_ECUDA;
  return contract_adjoint_batch(k, nvol, reinterpret_cast<const float2*>(d_in), reinterpret_cast<float2*>(d_out),
                                static_cast<cudaStream_t>(stream));
}

ctof_status ctof_forward_multiplexed(ctof_kernel k, const float* d_mu, float* d_y, void* stream) {
  if (!k || !d_mu || !d_y) return CTOF_EINVAL;
  if (k->n % 8 != 0) return CTOF_EUNSUPPORTED;
  DeviceGuard g(k->device);
  if (!g.ok) return CTOF_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CTOF_TRY(forward_impl(k, d_mu, d_y, st));
  return block_hadamard(d_y, k->nt, k->n, st);
}

ctof_status ctof_adjoint_multiplexed(ctof_kernel k, const float* d_y, float* d_vol, void* stream) {
  if (!k || !d_y || !d_vol) return CTOF_EINVAL;
  if (k->n % 8 != 0) return CTOF_EUNSUPPORTED;
  DeviceGuard g(k->device);
  if (!g.ok) return CTOF_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t meas = (size_t)k->nt * k->n * k->n;
  CTOF_CUDA_TRY(cudaMemcpyAsync(k->d_u1, d_y, meas * sizeof(float), cudaMemcpyDeviceToDevice, st));
  CTOF_TRY(block_hadamard(k->d_u1, k->nt, k->n, st));
  return adjoint_impl(k, k->d_u1, d_vol, st);
}

ctof_status ctof_reconstruct(ctof_kernel k, const float* d_m, const ctof_solver_params* params, float* d_mu,
                             ctof_report* report, void* stream) {
  if (!k || !d_m || !d_mu) return CTOF_EINVAL;
  CTOF_TRY(validate_params(params));
  DeviceGuard g(k->device);
  if (!g.ok) return CTOF_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t mbytes = (size_t)k->nt * k->n * k->n * sizeof(float);
  const size_t vbytes = (size_t)k->nz * k->n * k->n * sizeof(float);
  double lambda = 0.0;
  CTOF_CUDA_TRY(cudaMemcpyAsync(k->d_mstage, d_m, mbytes, cudaMemcpyDeviceToDevice, st));
  CTOF_TRY(solve_staged(k, params, &lambda, st));
  CTOF_CUDA_TRY(cudaMemcpyAsync(d_mu, k->d_vstage, vbytes, cudaMemcpyDeviceToDevice, st));
  if (report) return fill_report(k, params, lambda, report, st);
  return CTOF_OK;
}

ctof_status ctof_reconstruct_host(ctof_kernel k, const float* h_m, const ctof_solver_params* params, float* h_mu,
                                  ctof_report* report, void* stream) {
  if (!k || !h_m || !h_mu) return CTOF_EINVAL;
  CTOF_TRY(validate_params(params));
  DeviceGuard g(k->device);
  if (!g.ok) return CTOF_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t mbytes = (size_t)k->nt * k->n * k->n * sizeof(float);
  const size_t vbytes = (size_t)k->nz * k->n * k->n * sizeof(float);
  double lambda = 0.0;
  CTOF_CUDA_TRY(cudaMemcpyAsync(k->d_mstage, h_m, mbytes, cudaMemcpyHostToDevice, st));
  CTOF_TRY(solve_staged(k, params, &lambda, st));
  CTOF_CUDA_TRY(cudaMemcpyAsync(h_mu, k->d_vstage, vbytes, cudaMemcpyDeviceToHost, st));
  if (report) return fill_report(k, params, lambda, report, st);
  return take_device_status(k, st);
}

ctof_status ctof_reconstruct_batch_tikhonov(ctof_kernel k, int batch, const float* d_m, int precision,
                                            int refine_steps, double lambda_rel, float* d_mu, double* lambda_out,
                                            void* stream) {
  if (!k || !d_m || !d_mu || batch < 1 || batch > 4096) return CTOF_EINVAL;
  if (refine_steps < 0 || refine_steps > 8 || !finite_pos(lambda_rel)) return CTOF_EINVAL;
  if (precision != CTOF_FP32 && precision != CTOF_BF16 && precision != CTOF_FP8E4M3) return CTOF_EINVAL;
  if (precision != CTOF_FP32 && batch_tikhonov_smem_bytes(k->nt, k->nz) > 227 * 1024) return CTOF_EUNSUPPORTED;
  DeviceGuard g(k->device);
  if (!g.ok) return CTOF_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double lambda = lambda_rel * k->gram_max;
  if (lambda_out) *lambda_out = lambda;
  const size_t mvol = (size_t)k->nt * k->n * k->n, xvol = (size_t)k->nz * k->n * k->n;
  if (precision == CTOF_FP32) {
    // the plain FP32 path, one volume at a time (comparison baseline)
    ctof_solver_params prm{};
    prm.solver = CTOF_SOLVER_TIKHONOV;
    prm.tik_lambda_rel = lambda_rel;
    for (int b = 0; b < batch; ++b) {
      double lam = 0.0;
      CTOF_CUDA_TRY(cudaMemcpyAsync(k->d_mstage, d_m + b * mvol, mvol * sizeof(float), cudaMemcpyDeviceToDevice, st));
      CTOF_TRY(tikhonov_run(k, &prm, st, &lam));
      CTOF_CUDA_TRY(cudaMemcpyAsync(d_mu + b * xvol, k->d_vstage, xvol * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    return CTOF_OK;
  }
  const int ldm = ctof_round_up(batch * k->nt, 8), ldx = ctof_round_up(batch * k->nz, 8);
  const size_t b_sm = (size_t)k->nf * ldm * sizeof(float2), b_sx = (size_t)k->nf * ldx * sizeof(float2);
  const size_t b_in = (size_t)batch * (k->nt > k->nz ? k->nt : k->nz) * k->n * k->hp * sizeof(float2);
  const size_t need = ((b_sm + 255) & ~(size_t)255) + ((b_sx + 255) & ~(size_t)255) + b_in;
  if (need > k->batch_bytes) {
    CTOF_CUDA_TRY(cudaStreamSynchronize(st));
    if (k->d_batch) cudaFree(k->d_batch);
    k->d_batch = nullptr;
    k->batch_bytes = 0;
    if (cudaMalloc(&k->d_batch, need) != cudaSuccess) {
      cudaGetLastError();
      k->d_batch = nullptr;
      return CTOF_ENOMEM;
    }
    k->batch_bytes = need;
  }
  char* base = static_cast<char*>(k->d_batch);
  float2* spec_m = reinterpret_cast<float2*>(base);
  float2* spec_x = reinterpret_cast<float2*>(base + ((b_sm + 255) & ~(size_t)255));
  float2* inter = reinterpret_cast<float2*>(base + ((b_sm + 255) & ~(size_t)255) + ((b_sx + 255) & ~(size_t)255));
  CTOF_TRY(fft_forward_planes(k, d_m, batch * k->nt, k->n, k->n, k->n, inter, spec_m, ldm, st));
  CTOF_TRY(batch_tikhonov_prepare(k, lambda, st));
  CTOF_TRY(batch_tikhonov_contract(k, precision, batch, spec_m, ldm, spec_x, ldx, refine_steps, st));
  return fft_inverse_planes(k, spec_x, ldx, batch * k->nz, k->n, k->n, inter, d_mu, k->n, st);
}

ctof_status ctof_kernel_autotune(ctof_kernel k, void* stream) {
  if (!k) return CTOF_EINVAL;
  DeviceGuard g(k->device);
  if (!g.ok) return CTOF_ECUDA;
  k->tuned = 0;
  return autotune(k, static_cast<cudaStream_t>(stream));
}

ctof_status ctof_kernel_get_tuning(ctof_kernel k, int* h_pb4) {
  if (!k || !h_pb4) return CTOF_EINVAL;
  for (int i = 0; i < 4; ++i) h_pb4[i] = k->tune_pb[i];
  return k->tuned ? CTOF_OK : CTOF_EUNSUPPORTED;
}

ctof_status ctof_reconstruct_batch(int count, const ctof_kernel* ks, const float* const* d_m,
                                   const ctof_solver_params* params, float* const* d_mu, void* stream) {
  if (count < 1 || count > 4096 || !ks || !d_m || !d_mu) return CTOF_EINVAL;
  CTOF_TRY(validate_params(params));
  if (params->solver != CTOF_SOLVER_ADMM_TV) return CTOF_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (!ks[i] || !d_m[i] || !d_mu[i] || ks[i]->device != ks[0]->device) return CTOF_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ks[j] == ks[i]) return CTOF_EINVAL;  // a handle's workspace serves one problem at a time
  }
  DeviceGuard g(ks[0]->device);
  if (!g.ok) return CTOF_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < count; ++i) CTOF_TRY(autotune(ks[i], st));
  return batch_graph_run(count, ks, d_m, params, d_mu, st);
}

ctof_status ctof_set_wait_limit(ctof_kernel k, long long polls) {
  if (!k || polls < 0) return CTOF_EINVAL;
  k->max_polls = polls;
  return CTOF_OK;
}

ctof_status ctof_sync_status(ctof_kernel k, void* stream) {
  if (!k) return CTOF_EINVAL;
  DeviceGuard g(k->device);
  if (!g.ok) return CTOF_ECUDA;
  return take_device_status(k, static_cast<cudaStream_t>(stream));
}

ctof_status ctof_set_timing(ctof_kernel k, int enable) {
  if (!k || (enable != 0 && enable != 1)) return CTOF_EINVAL;
  k->timing = enable;
  return CTOF_OK;
}

ctof_status ctof_get_timing(ctof_kernel k, ctof_timing* out) {
  if (!k || !out) return CTOF_EINVAL;
  memset(out, 0, sizeof(*out));
  out->graph_kernel_nodes = k->graph_kernel_nodes;
  if (!k->graph || !k->graph_timing) return CTOF_EUNSUPPORTED;
  DeviceGuard g(k->device);
  const int iters = k->graph_iters;
  CTOF_CUDA_TRY(cudaEventSynchronize(k->events[4 * iters - 1]));
  for (int it = 0; it < iters; ++it) {
    float a = 0.f, b = 0.f, c = 0.f;
    CTOF_CUDA_TRY(cudaEventElapsedTime(&a, k->events[4 * it + 0], k->events[4 * it + 1]));
    CTOF_CUDA_TRY(cudaEventElapsedTime(&b, k->events[4 * it + 1], k->events[4 * it + 2]));
    CTOF_CUDA_TRY(cudaEventElapsedTime(&c, k->events[4 * it + 2], k->events[4 * it + 3]));
    out->contract_ms += a;
    out->t_side_ms += b;
    out->z_side_ms += c;
  }
  float tot = 0.f;
  CTOF_CUDA_TRY(cudaEventElapsedTime(&tot, k->events[0], k->events[4 * iters - 1]));
  out->iterations_ms = tot;
  out->contract_launches = iters;
  return CTOF_OK;
}

}  // extern "C"
