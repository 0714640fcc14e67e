/*
 * ctof.h -- C ABI of the GB300 confocal time-of-flight DOT library.
 *
 * The library implements the convolutional approximation of confocal
 * time-of-flight diffuse optical tomography (arXiv 2101.11680):
 *
 *   Eq. 2, Eq. 6   m = J mu : differential measurements are linear in the
 *                  absorption perturbation mu (Born approximation);
 *   Eq. 5          J(r_s, r_d, r_v, t) = Phi0(r_v - r_s, t) (*)_t R(r_d - r_v, t);
 *   Section 4      for confocal scans (source = detector) J is laterally
 *                  shift-invariant, so the forward model is a per-depth 2-D
 *                  convolution summed over depth (Eq. 9, Eq. 11):
 *                    m(x,y,t) = sum_z W_z(x,y,t) (*) mu_z(x,y).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Units: mm, ps, 1/mm.
 *  - Volumes mu are float32 [nz][ny][nx], measurements m are float32
 *    [nt][ny][nx]; x is the fastest axis; C order, contiguous.  Scan points
 *    sit on the lateral voxel-column centres (x_i = i dx, y_i = i dy).
 *    Voxel depth z_j = z_first + j dz; time bin k covers [k dt, (k+1) dt).
 *  - Pointers named d_* are device pointers (any allocation reachable by the
 *    device of the handle); h_* are host pointers.  The caller owns every
 *    data buffer; the library owns the handle and its workspaces.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls are stream-ordered and asynchronous unless they say
 *    otherwise; errors found on the host are returned at once.
 *  - A handle is not re-entrant: calls on one handle must not overlap on the
 *    device (issue them on one stream).  Separate handles are independent.
 *  - Every function returns ctof_status (0 = success); nothing throws
 *    across the ABI.  The GPU path has no CPU fallback: if no CUDA device is
 *    usable, calls that compute return CTOF_ECUDA.
 *  - Device-side waits (the tensor-core kernels' completion barriers) are
 *    bounded: one that runs out sets a sticky flag on the handle, lets the
 *    work in flight drain and stops its thread block, so that call's output
 *    is incomplete.  The flag is read and cleared by the next synchronising
 *    call on the handle (ctof_reconstruct with a report,
 *    ctof_reconstruct_host, ctof_learned_loss_grad, ctof_learned_train_step
 *    with a loss, ctof_sync_status), which then returns CTOF_ETIMEOUT.
 */
#ifndef CTOF_H
#define CTOF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CTOF_OK = 0,
  CTOF_EINVAL = -1,        /* bad argument: null pointer, size, optics */
  CTOF_ENOMEM = -2,        /* device allocation failed */
  CTOF_ECUDA = -3,         /* a CUDA runtime call failed */
  CTOF_ENONFINITE = -4,    /* a NaN/Inf was detected in an input or result */
  CTOF_ETIMEOUT = -5,      /* a bounded device wait gave up */
  CTOF_EUNSUPPORTED = -6   /* valid but not implemented (e.g. nx != ny) */
} ctof_status;

enum { CTOF_LINEAR = 0, CTOF_CIRCULAR = 1 };
enum { CTOF_SOLVER_ADMM_TV = 0, CTOF_SOLVER_TIKHONOV = 1, CTOF_SOLVER_FISTA_L1 = 2, CTOF_SOLVER_FISTA_L1_MUX = 3 };
enum { CTOF_KEEP_W = 1 }; /* ctof_build_kernel flag: retain the FP64 kernel table */
enum { CTOF_FP32 = 0, CTOF_BF16 = 1, CTOF_FP8E4M3 = 2 }; /* contraction precision */

/* Background optics of the homogeneous semi-infinite medium (Section 3,
 * "Analytical approximation"; the diffusion forms are the textbook
 * extrapolated-boundary ones).  mua >= 0, musp > 0, n >= 1. */
typedef struct {
  double mua_mm;   /* absorption coefficient [1/mm] */
  double musp_mm;  /* reduced scattering coefficient [1/mm] */
  double n;        /* refractive index of the medium */
  double z0_mm;    /* depth of the isotropic source; <= 0 selects 1/(mua+musp) */
  int clamp_r;     /* 1: clamp source/voxel/detector distances to >= min(dx,dy,dz)/2 */
} ctof_optics;

/* Confocal scan / voxel grid.  nx == ny is required; conv_mode selects the
 * lateral boundary: CTOF_LINEAR (zero-padded linear convolution, offsets in
 * [-(n-1), n-1], FFT size P = max(32, smallest power of two >= 2n)) or
 * CTOF_CIRCULAR (periodic, P = n, n a power of two).  Limits:
 * 4 <= nx <= 256 (linear), 32 <= nx <= 512 (circular), 1 <= nz <= 64,
 * 1 <= nt <= 1024, and one frequency class (its nt x nz block, H^-1 block
 * and vectors) must fit in the 227 KB of shared memory of one CTA: e.g.
 * nt <= 512 at nz = 64, nt <= 896 at nz = 32 (EUNSUPPORTED beyond). */
typedef struct {
  int nx, ny, nz, nt;
  double dx_mm, dy_mm, dz_mm;
  double z_first_mm;  /* depth of the first voxel layer (> 0) */
  double dt_ps;       /* time-bin width */
  int conv_mode;
} ctof_grid;

typedef struct ctof_kernel_s* ctof_kernel;

/* Read-only facts about a built kernel. */
typedef struct {
  int p;            /* lateral FFT size */
  int n_freq;       /* P * (P/2 + 1) half-plane frequencies */
  int n_class;      /* frequency classes sharing one W_hat matrix */
  int nt, nz;
  double scale;     /* max_f sigma_max(W_hat(f)) (the ADMM normalisation) */
  double gram_max_diag; /* max over f, j of (W_hat^T W_hat)_jj */
  size_t device_bytes;  /* device memory held by the handle */
  int admm_stages;      /* shared-memory stages of the pipelined ADMM x-update
                           kernel at this size (0: the fallback kernel runs) */
} ctof_kernel_info;

/* Solver choice and parameters.  ADMM_TV solves
 *   min_x 1/2 ||C K x - m||^2 + beta ||D x||_1,  x >= 0,  x = 0 off the scan
 * in units normalised by `scale` (K/scale has unit norm); Tikhonov solves
 * per lateral frequency (G + lambda I) x_hat = W_hat^T m_hat.  FISTA_L1 is the
 * paper's own solver (FISTA for the L1 problem of Eq. 8 with one weight per
 * depth, Eq. 10):
 *   min_x 1/2 ||A x - m||^2 + sum_z lam(z) ||x_z||_1,   A = C K / scale,
 * step 1, x_0 = 0, lam(z) = lam0 sigma(z) / max sigma with sigma(z) the DC
 * sensitivity of depth z (sqrt of the Gram diagonal at frequency 0), so that
 * deeper, fainter layers are thresholded less; lam0 = tv_beta (normalised
 * units) or, if tv_beta < 0, beta_rel * max|A^T m| / scale^2.  The report's
 * `beta` is lam0.  FISTA_L1_MUX solves the same problem for the multiplexed
 * composite operator of Eq. 12 (see ctof_forward_multiplexed): the measurement
 * passed is y = S m and A becomes S A with normalisation 8 scale; it needs a
 * lateral size that is a multiple of 8 (else EUNSUPPORTED). */
typedef struct {
  int solver;             /* CTOF_SOLVER_ADMM_TV, _TIKHONOV, _FISTA_L1 or _FISTA_L1_MUX */
  int iters;              /* ADMM / FISTA iterations (>= 1) */
  double rho;             /* ADMM penalty (> 0), e.g. 1 */
  double tv_beta;         /* TV weight (FISTA: lam0) in normalised units; < 0 selects
                             beta_rel * max|A^T m| / scale^2 */
  double beta_rel;        /* e.g. 1e-3 */
  double tik_lambda_rel;  /* lambda = tik_lambda_rel * gram_max_diag, e.g. 1e-3 */
} ctof_solver_params;

typedef struct {
  double scale;      /* normalisation used */
  double beta;       /* TV weight (FISTA: lam0) used, normalised units */
  double lambda;     /* Tikhonov lambda used */
  int iters_done;
} ctof_report;

/* Build the sensitivity kernel (Eq. 4-6 with the Section 4 convolutional
 * approximation): evaluates W[k][j][|oy|][|ox|] = dx dy dz * int_bin_k
 * (Phi0 (*)_t R)(rho, z_j, t) dt in FP64 on the device (closed-form time
 * convolution, 8-node x 4-piece Gauss-Legendre bin rule), transforms it to
 * the real lateral spectrum W_hat (FP64, stored FP32 per frequency class),
 * forms the per-frequency Gram matrices and the ADMM normal matrices (FP64
 * Cholesky, FP32 inverse).  Synchronous: returns when the handle is ready.
 * flags: 0 or CTOF_KEEP_W.  On success *out owns device memory until
 * ctof_kernel_destroy.  Errors: EINVAL (null pointer, non-positive sizes or
 * pitches, optics out of range), EUNSUPPORTED (nx != ny, sizes beyond the
 * limits above), ENOMEM, ECUDA. */
ctof_status ctof_build_kernel(const ctof_optics* optics, const ctof_grid* grid, int flags,
                              void* stream, ctof_kernel* out);

/* Emission side of the fluorescence mode (Section 5, simulator paragraph:
 * separate optical properties at the excitation and emission wavelengths,
 * and the response convolved with an exponential of the fluorescence
 * lifetime).  The refractive index is the excitation medium's. */
typedef struct {
  double mua_mm;   /* absorption at the emission wavelength [1/mm], >= 0 */
  double musp_mm;  /* reduced scattering at the emission wavelength [1/mm], > 0 */
  double tau_ps;   /* fluorescence lifetime [ps], >= 0 (0: instantaneous emission) */
} ctof_emission;

/* Build a fluorescence-mode kernel: as ctof_build_kernel, but with
 *   W[k][j][|oy|][|ox|] = dx dy dz * int_bin_k (Phi0_ex (*)_t L_tau (*)_t R_em)(rho, z_j, t) dt,
 * Phi0_ex the fluence of the excitation light (excitation optics: source
 * depth z0, extrapolated boundary), L_tau(t) = exp(-t/tau)/tau the
 * normalised lifetime density (a delta at tau = 0), R_em the surface flux
 * of the emission light (emission optics).  Evaluated in FP64 on the device
 * through the product of the three Laplace transforms (closed forms),
 * inverted with a 24-term fixed-Talbot rule at the bin edges; the bin
 * integral is the difference of the cumulative response at the two edges
 * (no time quadrature).  Everything downstream (spectrum, classes, Gram,
 * factorisations, every operator and solver) is the same as for an
 * absorption kernel.  The distance clamp of excitation->clamp_r applies to
 * both media.  Errors: as ctof_build_kernel, plus EINVAL for a null or
 * out-of-range emission (mua < 0, musp <= 0, tau < 0, non-finite). */
ctof_status ctof_build_kernel_fluorescence(const ctof_optics* excitation, const ctof_emission* emission,
                                           const ctof_grid* grid, int flags, void* stream, ctof_kernel* out);

/* Voxel-averaged kernel near the surface.  The time-domain forward model
 * integrates J mu over the volume (Section 3, Eq. of m(r_d, r_s, t)); with mu
 * constant on each voxel the exact weight of a voxel is the integral of J
 * over it, of which the centre value times the volume is the midpoint rule.
 * Near the surface and the source J varies strongly inside one voxel (the
 * paper notes the diffusion form is least reliable there, Section 3), so
 * the first `layers` depth layers take the voxel average, a tensor
 * Gauss-Legendre rule of `nodes` points per axis over the voxel
 * (centre +- dx/2, +- dy/2, +- dz/2; z_j is the layer centre). */
typedef struct {
  int layers;  /* 0..nz: depth layers, from the first, that are averaged (0 = none) */
  int nodes;   /* 1..8 Gauss-Legendre nodes per axis (1 = the centre value) */
} ctof_voxel_average;

/* General kernel build: absorption (emission == NULL) or fluorescence mode,
 * with (average != NULL) or without voxel averaging; otherwise as
 * ctof_build_kernel / ctof_build_kernel_fluorescence.  Cost of the table
 * build grows by nodes^3 on the averaged layers.  Errors: as those two,
 * plus EINVAL for layers outside [0, nz], nodes outside [1, 8], or
 * averaged layers reaching above the surface (z_first < dz/2 with
 * layers > 0). */
ctof_status ctof_build_kernel_ex(const ctof_optics* optics, const ctof_emission* emission,
                                 const ctof_voxel_average* average, const ctof_grid* grid, int flags,
                                 void* stream, ctof_kernel* out);

void ctof_kernel_destroy(ctof_kernel k);

ctof_status ctof_kernel_get_info(ctof_kernel k, ctof_kernel_info* info);

/* Copy the FP64 kernel table W[nt][nz][ny][nx] (non-negative offsets |oy|, |ox|;
 * for circular mode the table is [nt][nz][P/2+1][P/2+1]) to host memory.
 * Needs CTOF_KEEP_W at build time (else EUNSUPPORTED).  Synchronous. */
ctof_status ctof_kernel_get_w(ctof_kernel k, double* h_w);

/* Copy the frequency-class table to host: h_members[n_class][4] half-plane
 * frequency indices f = ky * (P/2+1) + kx of the frequencies sharing class c
 * (-1 = unused slot).  Synchronous. */
ctof_status ctof_kernel_get_classes(ctof_kernel k, int* h_members);

/* Copy W_hat as float32 [n_class][nt][nz] (real: the kernel is even) to
 * host memory.  Synchronous. */
ctof_status ctof_kernel_get_what(ctof_kernel k, float* h_what);

/* m = A mu (Eq. 11 with the linear or circular lateral boundary):
 * d_mu [nz][ny][nx] -> d_m [nt][ny][nx].  Asynchronous on `stream`. */
ctof_status ctof_forward(ctof_kernel k, const float* d_mu, float* d_m, void* stream);

/* vol = A^T m: d_m [nt][ny][nx] -> d_vol [nz][ny][nx].  Asynchronous. */
ctof_status ctof_adjoint(ctof_kernel k, const float* d_m, float* d_vol, void* stream);

/* Source multiplexing (Section 5, "Composite reconstruction algorithm",
 * Eq. 12): y = S A mu with S the 64 x 64 Sylvester Hadamard matrix (entries
 * +-1; the paper's 8 x 8 source array) acting, for every time bin, on each
 * 8 x 8 block of scan points taken row-major inside the block.  Layouts as
 * ctof_forward / ctof_adjoint; the lateral size must be a multiple of 8
 * (else EUNSUPPORTED).  The adjoint A^T S^T y (S^T = S) uses a workspace of
 * the handle.  Asynchronous. */
ctof_status ctof_forward_multiplexed(ctof_kernel k, const float* d_mu, float* d_y, void* stream);

/* Per-frequency contractions of Eq. 11 in the lateral Fourier domain for
 * nvol volumes at once, on frequency-major half-plane spectra (device
 * buffers, complex as interleaved float pairs, f = ky * (P/2+1) + kx):
 *   forward  d_out[v][f][t] = sum_z W_hat(f, t, z) d_in[v][f][z],
 *            d_in [nvol][n_freq][ldz], d_out [nvol][n_freq][ldt];
 *   adjoint  d_out[v][f][z] = sum_t W_hat(f, t, z) d_in[v][f][t],
 *            d_in [nvol][n_freq][ldt], d_out [nvol][n_freq][ldz];
 * ldz = nz rounded up to 8, ldt = nt rounded up to 8 (complex entries).
 * Input entries beyond nz / nt are ignored, output entries beyond them are
 * not written.  From 4 volumes on, 16 volumes and one frequency class form
 * one 128-wide tcgen05 GEMM (3xTF32, FP32-level accuracy); fewer volumes take
 * the FP32 CUDA-core path.  Asynchronous on `stream`; a device wait that runs
 * out is reported by the next synchronising call (ctof_sync_status).
 * Errors: EINVAL (null pointer, nvol < 1), ECUDA. */
ctof_status ctof_contract_forward_batch(ctof_kernel k, int nvol, const float* d_in, float* d_out, void* stream);
ctof_status ctof_contract_adjoint_batch(ctof_kernel k, int nvol, const float* d_in, float* d_out, void* stream);
ctof_status ctof_adjoint_multiplexed(ctof_kernel k, const float* d_y, float* d_vol, void* stream);

/* Reconstruct mu from m with the chosen solver: d_m [nt][ny][nx] ->
 * d_mu [nz][ny][nx].  If `report` is non-NULL the call synchronises the
 * stream and fills it; otherwise it is asynchronous.  ADMM runs as one
 * captured CUDA graph per handle (captured on first use).  Errors: EINVAL,
 * ECUDA; ENONFINITE (only with a report) if the result holds NaN/Inf. */
ctof_status ctof_reconstruct(ctof_kernel k, const float* d_m, const ctof_solver_params* params,
                             float* d_mu, ctof_report* report, void* stream);

/* As ctof_reconstruct but with HOST buffers h_m [nt][ny][nx] and
 * h_mu [nz][ny][nx]: copies in, reconstructs, copies out, and synchronises
 * the stream before returning.  Pinned host memory gives the fastest copies. */
ctof_status ctof_reconstruct_host(ctof_kernel k, const float* h_m, const ctof_solver_params* params,
                                  float* h_mu, ctof_report* report, void* stream);

/* Learned form (the paper has no learned component; this is an added
 * reconstruction option): an unrolled proximal-gradient solver with S stages
 *   g_s = A_n^T (A_n x_s - m_n),  z_s = x_s - eta_s g_s,
 *   x_{s+1} = z_s + mu0 f(z_s / mu0),
 * with A_n = A / scale, m_n = m / scale, mu0 = 0.01/mm, and f a 3-D CNN
 * shared by all stages: conv(1->16)+b, ReLU, conv(16->16)+b, ReLU,
 * conv(16->16)+b, ReLU, conv(16->1)+b, 3x3x3 taps, zero padding.  BF16
 * activations and weights, FP32 accumulation, FP32 masters.
 * x_0 is 0, or the per-frequency Tikhonov solution of m (options).  At
 * inference only, `dc_steps` data-consistency steps follow the last stage:
 *   x <- x - T(A x - m),  T = the per-frequency Tikhonov solve,
 * which remove what the data contradicts from the network's output (training
 * does not differentiate through them).
 * Parameters are a flat float array of ctof_learned_param_count(S) values:
 * w1 [16][1][27], b1 [16], w2 [16][16][27], b2 [16], w3 [16][16][27], b3 [16],
 * w4 [1][16][27], b4 [1], eta [S]; tap index (dz+1)*9 + (dy+1)*3 + (dx+1).
 * The kernel handle's lateral size must be a multiple of 16.  Loss (training):
 * mean over voxels of ((x_S - mu)/mu0)^2.  Batches are [batch][...] stacks of
 * the usual layouts.  A handle owns its workspace; not re-entrant. */
typedef struct ctof_learned_s* ctof_learned;
typedef struct {
  double x0_lambda_rel; /* > 0: x_0 = Tikhonov solution, lambda = x0_lambda_rel * max Gram diagonal; 0: x_0 = 0 */
  int dc_steps;         /* data-consistency steps after the last stage at inference (>= 0) */
  double dc_lambda_rel; /* relative Tikhonov lambda of those steps (> 0 when dc_steps > 0) */
} ctof_learned_options;
int ctof_learned_param_count(int stages);
/* opt may be NULL (x_0 = 0, no data-consistency steps). */
ctof_status ctof_learned_create(int stages, const float* h_params, const ctof_learned_options* opt,
                                ctof_learned* out);
void ctof_learned_destroy(ctof_learned net);
ctof_status ctof_learned_get_params(ctof_learned net, float* h_params);
/* Loss and its gradient w.r.t. the flat parameters for a batch (synchronous). */
ctof_status ctof_learned_loss_grad(ctof_learned net, ctof_kernel k, int batch, const float* d_m,
                                   const float* d_mu, double* h_loss, float* h_grad, void* stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on a batch; *h_loss (optional,
 * synchronising) receives the batch loss before the step. */
ctof_status ctof_learned_train_step(ctof_learned net, ctof_kernel k, int batch, const float* d_m,
                                    const float* d_mu, double lr, double* h_loss, void* stream);
/* Inference (stages, then the data-consistency steps):
 * d_m [batch][nt][n][n] -> d_mu [batch][nz][n][n].  Asynchronous. */
ctof_status ctof_learned_reconstruct(ctof_learned net, ctof_kernel k, int batch, const float* d_m,
                                     float* d_mu, void* stream);
/* Inference followed by the data-residual check that decides the ADMM
 * fallback: d_res[b] (device, batch doubles) = ||A mu_b - m_b||_2 / ||m_b||_2
 * with A the forward operator of Eq. 11 (m_b = 0 gives 0 for A mu_b = 0, else
 * +inf).  The check adds one batched forward contraction and, per member, one
 * inverse transform of the time planes that compares with m_b as it goes;
 * sums in FP64 of the FP32 values.  Asynchronous; the caller reads d_res and
 * reconstructs the members above its threshold another way (ctof_reconstruct).
 * Errors as ctof_learned_reconstruct, EINVAL for a null d_res. */
ctof_status ctof_learned_reconstruct_checked(ctof_learned net, ctof_kernel k, int batch, const float* d_m,
                                             float* d_mu, double* d_res, void* stream);

/* Batching form: ADMM reconstructions of `count` independent problems of
 * uneven sizes and optics (one handle each, distinct handles), d_m[i] ->
 * d_mu[i] with the layouts of ctof_reconstruct, all with `params`.  The batch
 * is one captured CUDA graph: per iteration, the x-update of every problem
 * whose class blocks fit the shared stages of the largest of them runs as one
 * persistent launch whose thread blocks take (problem, frequency class) items
 * from a device work queue; the other problems' x-updates and every problem's
 * FFT / TV stages run on forked streams.  The graph is kept and replayed
 * while the same handles, buffers and parameters come back (one cached batch
 * graph per process); results are bit-identical to reconstructing each
 * problem alone.  Handles not yet tuned are autotuned first (see
 * ctof_kernel_autotune), so the first call synchronises and must not be made
 * inside a stream capture.  The batch must not overlap other calls on its
 * handles.  Asynchronous after the first call; a bounded wait that runs out
 * in the queued launch is reported on the first queued handle (the wait limit
 * in force when the graph was made applies).  Errors: EINVAL (bad or
 * repeated handle, null buffer, handles on different devices), ENOMEM,
 * ECUDA. */
ctof_status ctof_reconstruct_batch(int count, const ctof_kernel* ks, const float* const* d_m,
                                   const ctof_solver_params* params, float* const* d_mu, void* stream);

/* Autotuner: times the column-FFT tile (32 or 16 columns of 8 or 16 planes) for each of the four column-pass shapes of an
 * ADMM iteration on this handle and keeps the fastest; the results are
 * bit-identical for every tile, only the speed changes.  Runs automatically
 * before the first ADMM graph capture of a handle.  Synchronous; not inside a
 * stream capture. */
ctof_status ctof_kernel_autotune(ctof_kernel k, void* stream);

/* The tuned tiles [T-side forward, T-side inverse, Z-side forward, Z-side
 * inverse] as tile codes: 8 / 16 = 32-column tiles of that many planes,
 * 108 / 116 = 16-column tiles of 8 / 16 planes; EUNSUPPORTED (defaults 16
 * reported) if not tuned yet. */
ctof_status ctof_kernel_get_tuning(ctof_kernel k, int* h_pb4);

/* Precision form: Tikhonov reconstruction of `batch` volumes that share the
 * kernel (the per-frequency regularised inverse of Eq. 7 applied to B
 * measurements at once).  d_m [batch][nt][ny][nx] -> d_mu [batch][nz][ny][nx].
 * CTOF_BF16 / CTOF_FP8E4M3: per frequency class and 16 volumes, b = W_hat^T
 * m_hat as one tcgen05 tensor-core GEMM with FP32 accumulation, the operands
 * split into terms whose sum reproduces the FP32 values (BF16: high +
 * remainder, three products; FP8 e4m3: s (q0 + q1/16 + q2/256) with s
 * mapping the block's largest magnitude to 448, per frequency class for
 * W_hat and per right-hand side for m_hat, six products); x0 = C b0 from the
 * first product alone, then `refine_steps` steps of
 * x += C (b - (G + lambda I) x) with C = (G + lambda I)^-1 from the FP64
 * Cholesky factor, those products in TF32 hi/lo on the tensor cores
 * (FP32-level).  CTOF_FP32: the plain FP32 per-volume path
 * (ctof_reconstruct with CTOF_SOLVER_TIKHONOV) for comparison.
 * lambda = lambda_rel * gram_max_diag; *lambda_out (optional) receives it.
 * The first BF16 / FP8 call for a lambda makes C, G + lambda I and their
 * tensor-core tables (per class ~4 nz^2 x 4 bytes plus 2 nz z4 x 4); the batch
 * workspace (spectra of batch x nt planes) is allocated on first use and
 * kept.  Asynchronous; a bounded device wait that runs out is reported by
 * ctof_sync_status.  Errors: EINVAL, EUNSUPPORTED (class block too large for
 * the kernel's shared memory), ENOMEM, ECUDA. */
ctof_status ctof_reconstruct_batch_tikhonov(ctof_kernel k, int batch, const float* d_m, int precision,
                                            int refine_steps, double lambda_rel, float* d_mu,
                                            double* lambda_out, void* stream);

/* m = A mu like ctof_forward, but allocation-free: every intermediate lives in
 * one fixed 32 MiB array inside the library image instead of the handle's
 * workspace, and the call makes no cudaMalloc/cudaFree or other allocating
 * call.  (The paper has no counterpart; this exists for callers that may not
 * allocate device memory at the point of the call: real-time acquisition
 * loops that must never wait on an allocator, and host frameworks or plugins
 * that own every device allocation and give the library only its inputs and
 * outputs.)  The handle must already be built.
 * The first call on a device resolves the array's device address with that
 * device current and keeps it for the life of the process; make that first
 * call before any stream capture begins.  The kept address does not survive
 * cudaDeviceReset (or any other teardown of the device's primary context):
 * do not call this entry point after one.
 * All calls share the array: calls that overlap on the GPU race and corrupt
 * each other; serialise them.  Grids whose intermediates exceed 32 MiB are
 * rejected with CTOF_EUNSUPPORTED (ctof_last_error_message gives the size).
 * Asynchronous on `stream`. */
ctof_status ctof_forward_static(ctof_kernel k, const float* d_mu, float* d_m, void* stream);

/* Device timing of the stages of the last ADMM reconstruction on a handle
 * (a profiling aid).  With ctof_set_timing(k, 1) the next captured ADMM graph
 * records CUDA events around each stage of every iteration: the per-class
 * x-update contraction, the T-side FFT chain and the Z-side FFT/TV chain.
 * ctof_get_timing waits for the last of those events and sums the stage
 * durations over the iterations; it returns EUNSUPPORTED (after filling
 * graph_kernel_nodes) if the current graph was captured without timing. */
typedef struct {
  double contract_ms;      /* sum over iterations of the x-update contraction */
  double t_side_ms;        /* sum of the T-side chains (K x -> v1/u1 -> c_hat) */
  double z_side_ms;        /* sum of the Z-side chains (x -> TV prox -> s_hat) */
  double iterations_ms;    /* first contraction start to last stage end */
  int contract_launches;   /* number of contraction launches summed */
  int graph_kernel_nodes;  /* kernel launches in one replay of the ADMM graph */
} ctof_timing;

ctof_status ctof_set_timing(ctof_kernel k, int enable);
ctof_status ctof_get_timing(ctof_kernel k, ctof_timing* out);

/* Bounded device waits (not from the paper: a safety property of this
 * library).  ctof_set_wait_limit sets how many times a kernel of this handle
 * polls a completion barrier before it gives up (default 2^24; 0 makes every
 * such wait give up at once, which tests use to exercise the error path).
 * polls < 0: EINVAL.  Host-only, takes effect at the next launch. */
ctof_status ctof_set_wait_limit(ctof_kernel k, long long polls);

/* Synchronises `stream`, then reads and clears the handle's sticky device
 * status: CTOF_ETIMEOUT if a bounded device wait of one of the handle's
 * kernels ran out since the last synchronising call (the output of that
 * call is incomplete), CTOF_OK otherwise. */
ctof_status ctof_sync_status(ctof_kernel k, void* stream);

const char* ctof_status_string(ctof_status s);

/* Text of the last CUDA runtime error seen by this thread inside the library
 * (empty if none).  The pointer stays valid until the next library call. */
const char* ctof_last_error_message(void);

#ifdef __cplusplus
}
#endif
#endif /* CTOF_H */
