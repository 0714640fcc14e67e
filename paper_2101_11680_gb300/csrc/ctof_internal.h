// Internal state of a ctof handle and the launchers each translation unit
// provides.  Not part of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "common.cuh"

// Device workspaces are carved from one allocation per handle.
struct ctof_kernel_s {
  ctof_optics optics;
  ctof_grid grid;
  int flags;
  int fluorescence;        // 1: W is the fluorescence-mode kernel with `emission`
  ctof_emission emission;
  ctof_voxel_average avg;  // layers = 0: centre values everywhere
  int device;

  // geometry
  int n;        // lateral scan size (nx == ny)
  int p;        // lateral FFT size
  int h;        // P/2 + 1 (half-plane width)
  int hp;       // kx pitch of the row-pass intermediates [row][hp][plane pitch]
  int nf;       // P * h half-plane frequencies
  int q;        // kernel-table extent per lateral axis (n linear, P/2+1 circular)
  int nt, nz;
  int z4;       // nz rounded up to a multiple of 4 (row pitch of W_hat and H^-1)
  int ldt, ldz; // frequency-major leading dims (complex) of T- and Z-side spectra
  int nclass;
  int symmetric;  // dx == dy: 8-fold lateral symmetry, classes hold up to 4 members

  double scale;     // max_f sigma_max(W_hat(f))
  double gram_max;  // max_{f,j} G_jj(f)
  double r_min;

  // one device allocation holds everything below
  void* d_base;
  size_t bytes;

  int* d_members;      // [nclass][4]
  float* d_lap;        // [nclass] 4 sin^2(pi a/P) + 4 sin^2(pi b/P)
  float* d_what;       // [nclass][nt][z4] (zero padding)
  double* d_gram;      // [nclass][nz][nz]
  float* d_hinv;       // [nclass][nz][z4]  (ADMM normal matrix inverse, normalised units)
  float* d_what_admm;  // W_hat in the ADMM kernel's block layout [nclass][tm/8][zm/8][64] (or null)
  float* d_hinv_admm;  // H^-1 in the same layout [nclass][zm/8][zm/8][64] (or null)
  float2* d_tw;        // FFT twiddle table (fft_twiddle_table layout)
  double* d_w;         // optional FP64 kernel table [nt][nz][q][q]

  float2* d_spec_t;    // [nf][ldt]
  float2* d_spec_t2;   // [nf][ldt]
  float2* d_spec_z;    // [nf][ldz]
  float2* d_spec_z2;   // [nf][ldz]
  float2* d_inter_t;   // [n][hp][round_up(nt, 16)]
  float2* d_inter_z;   // [p][hp][round_up(nz, 16)]
  float* d_u1;         // [nt][n][n]
  float* d_mstage;     // [nt][n][n]
  float* d_u2a;        // [3][nz][p][p]
  float* d_u2b;        // [3][nz][p][p]
  float* d_u3;         // [nz][p][p]
  float* d_xs;         // [nz][p][p]
  float* d_s;          // [nz][p][p]
  float* d_vstage;     // [nz][n][n]
  double* d_scalars;   // [16] device scalars (beta, max reductions, flags)
  int* d_flags;        // [4] sticky device status, cleared when read: [0] a bounded wait ran out
  long long max_polls; // polls before a device-side wait gives up (ctof_set_wait_limit)

  // Tikhonov cache: FP64 Cholesky factors of G + lambda I
  // Tikhonov inverses (G + lambda I)^-1 (FP64 Cholesky, stored FP32 [nclass][nz][z4])
  // for the two most recently used lambdas (separate allocations, made on first use)
  double tik_lambda[2];
  float* d_tik_hinv[2];
  int tik_last;  // slot used last

  // ADMM graph cache
  cudaGraphExec_t graph;
  int graph_iters;
  double graph_rho, graph_beta, graph_beta_rel;
  int graph_timing;
  int graph_kernel_nodes;

  // optional per-stage timing: 4 events per ADMM iteration, recorded inside the graph
  int timing;
  int n_events;
  cudaEvent_t* events;

  // precision form (batched Tikhonov): BF16 split tables, FP32 factors, batch workspace
  float* d_bt_cinv;    // [nclass][nz][z4] (G + lambda I)^-1 (one allocation holds the four below)
  float* d_bt_glam;    // [nclass][nz][z4] G + lambda I
  float* d_bt_sw;      // [nclass] FP8 scale of W_hat (max |W_hat| / 448)
  unsigned char* d_bt_tab;  // [nclass] C hi, C lo, G + lambda I hi, lo: BF16 [zn x zn] K-major tiles
  double bt_lambda;
  void* d_batch;       // batch spectra + row intermediates (one allocation)
  size_t batch_bytes;

  // autotuned column-pass plane tiles: [T fwd, T inv, Z fwd, Z inv]
  int tune_pb[4];
  int tuned;
  unsigned long long uid;  // unique per handle (batch graph cache key)
};

// Makes `dev` current for a scope and restores the previous device after it.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      ok = false;
      return;
    }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Default number of mbarrier polls before a device-side wait gives up.
constexpr long long CTOF_DEFAULT_MAX_POLLS = 1ll << 24;

// Synchronises `st`, then reads and clears the handle's sticky device status:
// CTOF_ETIMEOUT if a bounded device-side wait ran out since the last read.
ctof_status take_device_status(ctof_kernel_s* k, cudaStream_t st);

// ---- fft.cu -------------------------------------------------------------
// Complex elements of a row-pass intermediate for `rows` rows of `nplanes` planes.
size_t fft_inter_elems(const ctof_kernel_s* k, int nplanes, int rows);
// Twiddle table of the lateral FFTs for size p: its length and its host-side
// construction (FP64 roots rounded to FP32, in the layout the kernels stage).
int fft_twiddle_count(int p);
void fft_twiddle_table(int p, float2* out);

// Tiled tensor map (TMA descriptor) over `rank` dimensions of `elem_bytes`
// elements: dims innermost first, strides in bytes of dimensions 1 .. rank-1,
// box in elements, swizzle 0 / 32 / 64 / 128 bytes; out-of-range elements
// read as zero.  EINVAL for a misaligned base or stride, ECUDA when the driver
// rejects the map.
ctof_status ctof_encode_map(CUtensorMap* map, int elem_bytes, int rank, const void* base,
                            const unsigned long long* dims, const unsigned long long* strides_bytes,
                            const unsigned* box, int swizzle_bytes);
// Forward R2C of planes of real rows [nplanes][rows_in][ld_in] (first cols_in
// columns used, the rest of the P-wide row is zero) into frequency-major
// spectra out[f][ldf] (plane index fastest).  Zero rows beyond rows_in.
ctof_status fft_forward_planes(const ctof_kernel_s* k, const float* in, int nplanes, int rows_in,
                               int cols_in, int ld_in, float2* inter, float2* out, int ldf,
                               cudaStream_t st);
// Inverse C2R of frequency-major spectra in[f][ldf] into real rows
// out[nplanes][rows_out][ld_out] (first cols_out columns), scaled by 1/P^2.
ctof_status fft_inverse_planes(const ctof_kernel_s* k, const float2* in, int ldf, int nplanes,
                               int rows_out, int cols_out, float2* inter, float* out, int ld_out,
                               cudaStream_t st);
// Column passes alone (used by the fused ADMM chains).
ctof_status fft_cols_forward(const ctof_kernel_s* k, const float2* inter, int nplanes, int rows_in,
                             float2* out, int ldf, cudaStream_t st);
ctof_status fft_cols_inverse(const ctof_kernel_s* k, const float2* in, int ldf, int nplanes,
                             int rows_out, float2* inter, cudaStream_t st);
ctof_status fft_cols_forward_pb(const ctof_kernel_s* k, const float2* inter, int nplanes, int rows_in,
                                float2* out, int ldf, int pb, cudaStream_t st);
ctof_status fft_cols_inverse_pb(const ctof_kernel_s* k, const float2* in, int ldf, int nplanes,
                                int rows_out, float2* inter, int pb, cudaStream_t st);
ctof_status fft_rows_forward(const ctof_kernel_s* k, const float* in, int nplanes, int rows,
                             int cols_in, int ld_in, float2* inter, cudaStream_t st);
ctof_status fft_rows_inverse(const ctof_kernel_s* k, const float2* inter, int nplanes, int rows,
                             int cols_out, float* out, int ld_out, cudaStream_t st);
// ADMM T side: inverse rows of K x (crop) -> v1/u1 update -> forward rows of
// the correction c, in place in `inter` ([nt][n][hp]).
ctof_status fft_rows_admm_t(const ctof_kernel_s* k, float2* inter, const float* m, float* u1,
                            float inv_scale, float rho, cudaStream_t st);
// Learned-solver T side, in place on inter [n][kx][nt planes]: inverse rows,
// crop to the scan, c = Kx - m (Kx when m is null), forward rows of c.
ctof_status fft_rows_resid_t(const ctof_kernel_s* k, float2* inter, const float* m, cudaStream_t st);
// Inverse rows without a store: acc[0] += sum (z - ref)^2, acc[1] += sum ref^2
// over the first cols_out columns (ref laid out like fft_rows_inverse's out).
ctof_status fft_rows_inverse_norm(const ctof_kernel_s* k, const float2* inter, int nplanes, int rows, int cols_out,
                                  const float* ref, int ld_ref, double* acc, cudaStream_t st);

// ---- contract.cu --------------------------------------------------------
// shared memory the contraction kernels need at this size (single-buffered worst case)
size_t contract_smem_bytes(int nt, int nz);
ctof_status contract_forward(const ctof_kernel_s* k, const float2* in_z, float2* out_t, cudaStream_t st);
// nvol volumes sharing the kernel; spectra [nvol][nf][ld] (W_hat read once per class for all)
// Batched forward / adjoint on the tcgen05 tensor cores (contract_tc.cu):
// 16 volumes x one frequency class = one 128-wide GEMM, 3xTF32.
ctof_status contract_tc_forward(const ctof_kernel_s* k, int nvol, const float2* in_z, float2* out_t,
                                cudaStream_t st);
ctof_status contract_tc_adjoint(const ctof_kernel_s* k, int nvol, const float2* in_t, float2* out_z,
                                cudaStream_t st);
// The same with the Z-side spectra of all volumes interleaved per frequency
// (the output layout of one plane-batched FFT over nvol * nz planes): volume
// v's plane z at column v * nz + z of row f, row pitch ldzb (a multiple of 8,
// >= nvol * nz).  nz must be even (16-byte aligned volume rows); T-side
// spectra stay [v][f][ldt].  EINVAL otherwise.
ctof_status contract_tc_forward_zb(const ctof_kernel_s* k, int nvol, const float2* in_z, int ldzb, float2* out_t,
                                   cudaStream_t st);
ctof_status contract_tc_adjoint_zb(const ctof_kernel_s* k, int nvol, const float2* in_t, float2* out_z, int ldzb,
                                   cudaStream_t st);
ctof_status contract_tikhonov_zb(const ctof_kernel_s* k, int nvol, const float* hinv, const float2* m_hat,
                                 float2* x_hat, int ldzb, cudaStream_t st);
ctof_status contract_forward_batch(const ctof_kernel_s* k, int nvol, const float2* in_z, float2* out_t,
                                   cudaStream_t st);
ctof_status contract_adjoint_batch(const ctof_kernel_s* k, int nvol, const float2* in_t, float2* out_z,
                                   cudaStream_t st);
ctof_status contract_tikhonov_batch(const ctof_kernel_s* k, int nvol, const float* hinv, const float2* m_hat,
                                    float2* x_hat, cudaStream_t st);
ctof_status contract_adjoint(const ctof_kernel_s* k, const float2* in_t, float2* out_z, cudaStream_t st);
ctof_status contract_admm(const ctof_kernel_s* k, const float2* c_hat, const float2* s_hat,
                          float2* x_hat, float2* kx_hat, float inv_scale, cudaStream_t st);
ctof_status contract_tikhonov(const ctof_kernel_s* k, const float* hinv, const float2* m_hat,
                              float2* x_hat, cudaStream_t st);
size_t contract_admm_smem_bytes(int nt, int nz, int nbuf);
// Floats per class of the pipelined ADMM kernel's W_hat (which = 0) or H^-1
// (which = 1) copy; 0 when that kernel does not apply at this size.
size_t contract_admm_pipe_floats(int nt, int nz, int which);
// Stages of the pipelined ADMM kernel at this size (0: the fallback kernel).
int contract_admm_pipe_stages(int nt, int nz);
// Fill the pipelined kernel's copies from d_what / d_hinv (after the build).
ctof_status contract_admm_prepare(ctof_kernel_s* k, cudaStream_t st);

// Batched x-update: the problems of a batch whose class blocks fit two shared
// stages of the largest among them, in one persistent launch fed by a device
// work queue.  `members` lists their indices in the batch (queue order); the
// other problems keep their own contract_admm launch.  Timeouts are reported
// on the first queued problem's handle.
struct AdmmQueue {
  int nprob = 0, total = 0, stage_bytes = 0, stages = 0, o_scr = 0, zm_max = 0, smem = 0, nsm = 152;
  void* d_mem = nullptr;  // problem table, then the queue counter
  int* flag = nullptr;
  long long max_polls = 0;
  std::vector<int> members;
};
ctof_status admm_queue_build(int count, ctof_kernel_s* const* ks, AdmmQueue* out);
ctof_status admm_queue_launch(const AdmmQueue& q, cudaStream_t st);
void admm_queue_free(AdmmQueue* q);

// ---- batch_tikhonov.cu ----------------------------------------------------
size_t batch_tikhonov_smem_bytes(int nt, int nz);
ctof_status batch_tikhonov_prepare(ctof_kernel_s* k, double lambda, cudaStream_t st);
ctof_status batch_tikhonov_contract(const ctof_kernel_s* k, int precision, int batch, const float2* m_hat, int ldm,
                                    float2* x_hat, int ldx, int refine, cudaStream_t st);

// ---- build.cu ----------------------------------------------------------
ctof_status build_kernel_tables(ctof_kernel_s* k, cudaStream_t st);
ctof_status build_tikhonov_factors(ctof_kernel_s* k, int slot, double lambda, cudaStream_t st);
// (G + lambda I)^-1 for an absolute lambda, made on first use (two cached lambdas).
ctof_status tikhonov_inverse(ctof_kernel_s* k, double lambda, const float** hinv, cudaStream_t st);

// ---- admm.cu ------------------------------------------------------------
ctof_status admm_tv_stencil(const ctof_kernel_s* k, const float* x, const float* u2_old,
                            float* u2_new, float* u3, float* s, const double* beta_dev,
                            float rho, float* out_crop, cudaStream_t st);
ctof_status reduce_max_abs(const float* v, size_t count, double* out_dev, cudaStream_t st);
ctof_status admm_set_beta(double* scalars, double beta_fixed, double beta_rel, double inv_scale2,
                          cudaStream_t st);
ctof_status check_finite(const float* v, size_t count, int* flag_dev, cudaStream_t st);
// FISTA (Eq. 8, Eq. 10): per-depth weights from lam0 = scalars[0], r -= m, and one step
// (x holds x_{k-1} on entry and x_k on exit; y becomes the next extrapolated point).
ctof_status fista_lambda(const ctof_kernel_s* k, const double* scalars, float* lam, cudaStream_t st);
// In place, [planes][n][n]: every 8 x 8 block of scan points <- H_64 times it (n % 8 == 0).
ctof_status block_hadamard(float* v, int planes, int n, cudaStream_t st);
ctof_status fista_sub_meas(float* r, const float* m, size_t count, cudaStream_t st);
ctof_status fista_step(float* y, const float* g, float* x, const float* lam, float beta, float inv_s2, int plane,
                       size_t count, cudaStream_t st);
