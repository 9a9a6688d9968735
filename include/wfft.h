/*
 * wfft -- GB300-native implicit FFT elastodynamics (Sancho, Segurado et al.,
 * "FFT-based simulation of elastic waves", arXiv 2211.08263).
 *
 * C ABI of the CUDA library libwfft.so.  Every operation of the hot path runs
 * in hand-written sm_103a kernels behind these calls: batched radix-staged
 * real FFTs fused with the i*xi gradient / divergence multiplies, the
 * pointwise sigma = C(x):eps kernel, the closed-form reference-medium
 * preconditioner, warp-shuffle FP64 reductions, the Newmark predictor /
 * corrector and the prescribed-displacement (Dirichlet) region.
 *
 * Array conventions (all calls):
 *   - a grid is N1 x N2 x N3 voxels (N3 = 1 for ndim = 2, plane strain);
 *     voxel centres x = h (1/2 + idx) (Sec. 2.2.3);
 *   - scalar fields are C-ordered [N3][N2][N1] (x fastest), vector fields
 *     [c][N3][N2][N1] with c = ndim components, FP64 unless stated;
 *   - a stiffness is 21 FP64 Voigt upper-triangle values, order
 *     (11,22,33,23,13,12) x (11,22,33,23,13,12) row by row (C11 C12 ... C16
 *     C22 ... C66), C_IJ = C_ijkl with no factor 2; 2-D uses the in-plane
 *     entries of (11,22,12);
 *   - a Dirichlet mask is uint8 [c][N3][N2][N1], 1 = prescribed DOF.
 * Ownership: wfft_create copies every host array into device memory owned
 * by the handle; calls taking `*_dev` pointers read/write caller-owned
 * device memory and never free it.  All device work is issued on the stream
 * given at creation (NULL = the legacy default stream); calls that return
 * host data synchronise that stream.  A handle must be used by one host
 * thread at a time.
 * Errors: every call returns a WFFT_* status; no exception crosses the ABI.
 * wfft_last_error() gives the text of the last failure on a handle.
 */
#ifndef WFFT_H
#define WFFT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define WFFT_API __attribute__((visibility("default")))
#else
#define WFFT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define WFFT_OK 0
#define WFFT_EINVAL 1        /* bad sizes or arguments, non-SPD stiffness, rho <= 0, dt <= 0, all DOFs masked */
#define WFFT_ENOMEM 2        /* device or host allocation failed */
#define WFFT_ECUDA 3         /* a CUDA runtime call failed */
#define WFFT_ENOTCONV 4      /* Krylov solve hit maxit; the step is not committed, state unchanged */
#define WFFT_ENUMERIC 5      /* NaN/Inf or a non-positive curvature p.Ap in the solve; step not committed */
#define WFFT_ETIMEOUT 6      /* iteration watchdog fired; step not committed */
#define WFFT_EUNSUPPORTED 7  /* axis with two prime factors > 7 (or one > 127) or too long for the tiles, or N2 = N3 = 1 */

/* arithmetic of the Krylov solve */
#define WFFT_FP64 0   /* everything FP64 */
#define WFFT_MIXED 1  /* FP32 FFTs/stress/preconditioner inside PCG, FP64 dots, FP64 true-residual
                         refinement and FP64 Newmark state */

/* warm start of the solve of each step */
#define WFFT_WARM_PREV 0     /* x0 = u_{n-1} (the paper's choice) */
#define WFFT_WARM_TAYLOR 1   /* x0 = u + dt v + dt^2/2 a */
#define WFFT_WARM_LEARNED 2  /* x0 = u + dt v + dt^2/2 a + s y, y = network prediction (wfft_set_model) */

typedef struct wfft_handle wfft_handle;

typedef struct {
  int ndim;      /* 2 (plane strain, n[2] must be 1) or 3 */
  int n[3];      /* N1, N2, N3 */
  double h[3];   /* voxel size per axis (m); L_i = N_i h_i */
} wfft_grid;

typedef struct {
  int precision;     /* WFFT_FP64 or WFFT_MIXED */
  double tol;        /* relative residual target (see wfft_step) */
  int maxit;         /* cap on Krylov iterations per solve (FP64) or per inner solve (mixed) */
  int warm_start;    /* WFFT_WARM_* */
  double inner_tol;  /* mixed: relative reduction of each FP32 inner solve */
  int max_sweeps;    /* mixed: cap on FP64 refinement sweeps per solve */
  int check_every;   /* iterations between host reads of the device convergence flag */
  int watchdog_iters;/* hard cap on iterations per step, across sweeps (0 = 4*maxit) */
  int use_graphs;    /* 1: each block of check_every PCG iterations is one CUDA graph launch (captured
                        once per handle on an internal stream; not while profiling is on); 0: plain launches */
  double inner_floor;/* mixed: an FP32 inner solve also stops once its residual is below
                        inner_floor * tol * ref (the outer target), so the last sweep does not
                        overshoot it; 0 = off.  The FP64 residual still decides convergence. */
  int incr_resid;    /* mixed: 1 = the residual after a sweep that started from a full FP64
                        residual evaluation may be formed incrementally, b - (A x + xc A d): A x
                        the FP64 product kept from that evaluation, A d the FP32 product of the
                        sweep's correction d, accumulated in FP64.  Taken only when the rounding
                        estimate 8 * 2^-24 * lam_max(A) * ||xc d|| (lam_max bounded from C, rho,
                        the grid and theta, see wfft_operator_bound; 8 is eleven times the
                        largest measured ratio of the FP32 product's error to 2^-24 lam_max ||d||)
                        is at most tol * ref / 4; the estimate is added to ||r|| in the
                        convergence test.  At most one such update follows a full evaluation.
                        0 = every residual is a full FP64 application. */
} wfft_options;

typedef struct {
  int status;          /* WFFT_* of the step */
  int iters;           /* Krylov iterations = operator applications q = P A p (FP32 ones in mixed) */
  int outer_applies;   /* FP64 true-residual applications (mixed: one per sweep; FP64: 1) */
  int sweeps;          /* mixed: refinement sweeps */
  double ref;          /* ||P(b - A x_Gamma)||_2, x_Gamma = U on Gamma, 0 elsewhere */
  double rel_res;      /* final ||P(b - A x)||_2 / ref (FP64 true residual in mixed mode) */
  double reaction[3];  /* sum over the grid of rho a_n per component = total force on Gamma */
  double ms;           /* device time of the call (CUDA events) */
  int incr_resids;     /* mixed: incremental residual evaluations (see wfft_options.incr_resid) */
  double energy;       /* E_n = 1/2 sum_x rho |v_n|^2 + 1/2 sum_x eps_n : C : eps_n of the committed state
                          (sums over voxels, no cell volume; the energy of the Newmark energy identity,
                          Eq. Newmark with beta = 1/4, gamma = 1/2).  Implicit steps form the strain part
                          from the step's own sums, u.K u = sum_j U_j F_j - sum_x rho u_n . a_n with F_j
                          the reaction (A u_n = b + theta f, f on Gamma), exact up to the solver residual;
                          explicit steps from K u_n itself.  0 for a step that is not committed. */
} wfft_step_info;

/* Fill *opt with defaults: FP64, tol 1e-10, maxit 1000, WARM_PREV, inner_tol 1e-5,
   max_sweeps 20, check_every 4, use_graphs 1, inner_floor 0.5, incr_resid 1. */
WFFT_API int wfft_default_options(wfft_options* opt);

/*
 * Create a solver for one periodic heterogeneous medium (Alg. 2 "Data",
 * Sec. 2.2.3).
 *   grid      : dimensions and voxel sizes.
 *   C         : host, nphase x 21 Voigt stiffnesses (phase != NULL) or
 *               V x 21 per-voxel stiffnesses (phase == NULL).
 *   phase     : host uint16 [N3][N2][N1] phase id per voxel, or NULL.
 *   nphase    : rows of C / rho when phase != NULL (ignored otherwise).
 *   rho       : host, nphase (or V) densities, > 0.
 *   mask      : host uint8 [c][N3][N2][N1], 1 = prescribed DOF (Gamma), may be
 *               NULL (no prescribed region); must leave at least one free DOF.
 *   dt, beta, gamma : Newmark constants (Eq. Newmark); dt > 0, beta > 0; or beta = 0 with
 *                     gamma = 1/2 (FP64 only): an explicit-scheme handle, stepped by
 *                     wfft_explicit_step (wfft_step / wfft_solve / wfft_batch_step: EINVAL).
 *   opt       : options (NULL = defaults).
 *   stream    : cudaStream_t cast to void* (NULL = legacy default stream).
 *   out       : receives the handle (owned by the caller, free with wfft_destroy).
 * The volume averages Cbar and rho_bar of the preconditioner (Eq. precond,
 * Eq. acous) and the lifting fields used by the stopping test are computed
 * here.  Returns WFFT_EINVAL / WFFT_EUNSUPPORTED / WFFT_ENOMEM / WFFT_ECUDA.
 * Axis lengths: prime factors 2, 3, 5, 7 and at most one other prime P <= 127 (the
 * paper's odd grids, e.g. 129 = 3 x 43 and 1025 = 5^2 x 41, Sec. 4.1); P is taken by a
 * direct P-point DFT stage ((P - 1) / 2 paired terms per two outputs) ahead of the radix
 * stages; each axis must also fit the tiles of the passes (EUNSUPPORTED otherwise).
 * The state starts at rest (u = v = a = 0).
 */
WFFT_API int wfft_create(const wfft_grid* grid, const double* C, const uint16_t* phase, int nphase,
                const double* rho, const uint8_t* mask, double dt, double beta, double gamma,
                const wfft_options* opt, void* stream, wfft_handle** out);

/* Free every device and host resource of the handle (NULL is a no-op). */
WFFT_API void wfft_destroy(wfft_handle* h);

/* Text of the last error on h; with h NULL, of the last failed call without a handle
   made by the calling host thread. */
WFFT_API const char* wfft_last_error(const wfft_handle* h);

/* Replace the Newmark state (u_{n}, v_{n}, a_{n}) from host arrays [c][N3][N2][N1] and the
   step counter n.  Any pointer may be NULL (that field is set to 0). */
WFFT_API int wfft_set_state(wfft_handle* h, const double* u, const double* v, const double* a, long long n);

/* Copy the state to host arrays (any pointer may be NULL) and return the step counter in *n. */
WFFT_API int wfft_get_state(const wfft_handle* h, double* u, double* v, double* a, long long* n);
/* Asynchronous download of the state (u, v, a; NULL entries skipped) to host memory
   (pinned memory for overlap; pageable memory works but is staged): the copies are
   ordered after all work issued so far on the handle's stream and run on an internal
   copy stream, so they overlap the next wfft_step's solve; the next call that writes
   the state (the corrector of wfft_step / wfft_green_step / wfft_batch_step, the
   explicit predictor, wfft_set_state*) waits for them on the device.  The host buffers
   must stay valid until wfft_download_wait returns. */
WFFT_API int wfft_download_async(wfft_handle* h, double* u, double* v, double* a);
/* Blocks until the latest wfft_download_async of h has completed. */
WFFT_API int wfft_download_wait(wfft_handle* h);

/* Device-pointer variants (caller-owned FP64 device arrays, same layout). */
WFFT_API int wfft_set_state_dev(wfft_handle* h, const double* u, const double* v, const double* a, long long n);
WFFT_API int wfft_get_state_dev(const wfft_handle* h, double* u, double* v, double* a);

/*
 * Advance one beta-Newmark step (the loop body of Alg. 2):
 *   predictor  u~ = u + dt v + dt^2 (1/2 - beta) a,  b = rho u~   (Eq. Fourier_ND_b)
 *   solve      u_n|_Gamma = U(t_n) (component j of a prescribed DOF takes U[j]) and
 *              (A u_n - b) = 0 on every free DOF, A of Eq. Fourier_ND_A, by PCG
 *              with the preconditioner of Eq. precond on the masked system; this
 *              is the discrete solution that the Green's-matrix construction of
 *              Eqs. lin_prob1 .. L-determination_ND reaches;
 *              stop when ||P(b - A u)||_2 <= tol * ref;
 *   corrector  a_n = (u_n - u~)/(beta dt^2), v_n = v + dt((1-gamma) a + gamma a_n).
 *   U    : host, 3 values U(t_n) (the third ignored in 2-D).
 *   info : may be NULL.
 * On WFFT_ENOTCONV / WFFT_ENUMERIC / WFFT_ETIMEOUT the state is unchanged.
 */
WFFT_API int wfft_step(wfft_handle* h, const double U[3], wfft_step_info* info);

/*
 * One constrained solve A x = b (no Newmark update): x holds the warm start on
 * entry and its prescribed DOFs (mask = 1) keep their entry values; on exit x
 * solves (A x - b) = 0 on the free DOFs to ||P(b - A x)|| <= tol * ref.
 * b, x: host FP64 [c][N3][N2][N1].  tol <= 0 / maxit <= 0 take the handle's options.
 */
WFFT_API int wfft_solve(wfft_handle* h, const double* b, double* x, double tol, int maxit, wfft_step_info* info);

/*
 * Operator application q = A p (Eq. Fourier_ND_A), or q = P A p when masked != 0
 * (P zeroes the prescribed DOFs).  p_dev, q_dev: caller-owned device arrays
 * [c][N3][N2][N1] of double (precision WFFT_FP64) or float (WFFT_MIXED = the
 * FP32 kernels).  Asynchronous on the handle's stream.
 */
WFFT_API int wfft_apply(wfft_handle* h, int precision, const void* p_dev, void* q_dev, int masked);

/*
 * Preconditioner z = M r, M^(xi) = (theta K(xi) + rho_bar I)^-1 (Eq. precond,
 * Eq. acous), or z = P M r when masked != 0.  Same conventions as wfft_apply.
 */
WFFT_API int wfft_precond(wfft_handle* h, int precision, const void* r_dev, void* z_dev, int masked);

/*
 * Forward 3-D real FFT of `ncomp` (1..6) real fields (dir = +1 ... see below) in the
 * library's spectral layout, for testing the transforms against the DFT
 * definition (Eq. Fourier_derivatives uses the DFT of Sec. 2.1.3):
 *   dir = -1: in_dev real [ncomp][N3][N2][N1] -> out_dev complex (interleaved re,im)
 *             [ncomp][N3][N2][pitch], X[k] = sum_x f(x) exp(-2 pi i k.x/N), kx < N1/2+1;
 *   dir = +1: the unnormalised inverse (complex -> real), in the same layouts.
 * `pitch` (>= N1/2+1) is returned by wfft_spectral_pitch.  Asynchronous.
 */
WFFT_API int wfft_rfft3(wfft_handle* h, int precision, int dir, int ncomp, const void* in_dev, void* out_dev);
WFFT_API int wfft_spectral_pitch(const wfft_handle* h, int* pitch);

/*
 * Advance n independent handles by one step each (the batched workload of
 * uneven grids): the handles' solves are interleaved so that each pass of the
 * Krylov iteration is one grouped launch over all still-unconverged handles.
 * Handles must share precision and stream.  U: host n x 3.  infos: n entries or NULL.
 * Returns the first non-OK status (each info carries its own).
 */
WFFT_API int wfft_batch_step(wfft_handle** hs, int n, const double* U, wfft_step_info* infos);

/*
 * Learned warm start.  Not part of the paper's method: the paper starts each
 * step's Krylov solve from u_{n-1}.  A small network predicts the part of the
 * next displacement that the Taylor extrapolation misses, and the prediction
 * only changes the initial guess: the same stopping test (see wfft_step) still
 * decides when a step has converged.
 *
 * Network: four periodic 3x3x3 convolutions 16 -> H -> H -> H -> 3 with ReLU
 * after the first three, H = 16 or 32; BF16 weights and activations, FP32
 * accumulation and biases.  Inputs per voxel (channels-last, 16): dt v / s (3),
 * (dt^2/2) a / s (3), U(t_n) - (u + dt v + dt^2/2 a) on the prescribed DOFs / s
 * (3), prescribed indicator, rho / rho_bar - 1, C_11 / C_bar_11 - 1,
 * C_22 / C_bar_22 - 1, C_33 / C_bar_33 - 1, (C_44 + C_55 + C_66) / mean - 1,
 * (C_12 + C_13 + C_23) / mean - 1 (2-D: the in-plane entries, absent ones 0),
 * with s = sqrt(mean over DOFs of (dt v)^2 + (dt^2/2 a)^2, plus the prescribed
 * increments squared / (c V)).  Output y (3 channels): the warm start is
 * x0 = u + dt v + dt^2/2 a + s y on the free DOFs and U(t_n) on Gamma; the
 * training target is (u_n - u - dt v - dt^2/2 a) / s = beta dt^2 (a_n - a_{n-1}) / s.
 *
 * Model blob (host memory, native byte order): 8 int32 {magic 0x314E4657,
 * version 1, layers 4, cin 16, hidden H, cout 3, cout_pad 16, 0}, then per layer
 * l = 1..4 the FP32 weights W[27][cout_l][cin_l] (offset o = 9 (dz+1) +
 * 3 (dy+1) + (dx+1), output voxel x reads input voxel x + (dx, dy, dz) mod N)
 * followed by the FP32 biases b[cout_l]; cout_4 = 16 (only the first 3 are used).
 */
/* Kernel of the network's forward convolutions (process-wide): 0 (default) = the tcgen05
   kernel (5th-generation tensor cores, FP32 accumulators in tensor memory) for H = 32 on
   grids with N1 % 8 == 0 and N2 % 16 == 0, the mma.sync kernel otherwise; 1 = the mma.sync
   kernel everywhere (for comparing the two).  Returns the previous setting, or -1 for an
   unknown kind.  A tcgen05 convolution whose bounded wait expires makes the step that ran
   it return WFFT_ETIMEOUT without committing (wfft_net_forward / wfft_trainer_fit: the same
   status). */
WFFT_API int wfft_net_conv_kernel(int kind);
/* Bytes of a model blob of hidden width H (0 unless H is 16 or 32). */
WFFT_API size_t wfft_model_bytes(int hidden);
/* Seeded initial model: He-normal weights for layers 1-3, zero last layer (so the
   untrained network reproduces the Taylor warm start exactly).  bytes must equal
   wfft_model_bytes(hidden). */
WFFT_API int wfft_model_init(int hidden, unsigned long long seed, void* blob, size_t bytes);
/* Load a model into a handle (copied; the blob may be freed afterwards) for
   warm_start = WFFT_WARM_LEARNED.  blob = NULL with bytes = 0 unloads.  Allocates
   (16 + 2 H) * 2 bytes per voxel of work buffers.  EINVAL on a malformed blob. */
WFFT_API int wfft_set_model(wfft_handle* h, const void* blob, size_t bytes);

/* GPU training of the warm-start network on trajectories of the method itself. */
typedef struct wfft_trainer wfft_trainer;
/* Trainer on the current device starting from a model blob, issuing its work on
   cuda_stream (NULL = default stream).  Keeps FP32 master parameters and Adam moments. */
WFFT_API int wfft_trainer_create(const void* blob, size_t bytes, void* cuda_stream, wfft_trainer** out);
/* Advance handle h by nsteps steps (U: nsteps x 3, as wfft_step) and keep one
   training pair per step (features of the state before the step, target after it),
   (16 * 2 + 4 * 4) bytes per voxel per step on the device.  infos (nsteps entries,
   optional) receives each step's wfft_step_info.  A failing step stops the
   collection with its status; the pairs of the earlier steps are kept. */
WFFT_API int wfft_trainer_collect(wfft_trainer* t, wfft_handle* h, const double* U, int nsteps,
                                  wfft_step_info* infos);
/* Number of training pairs collected so far. */
WFFT_API long long wfft_trainer_samples(const wfft_trainer* t);
/* epochs passes over the pairs in seeded random order; Adam (beta1 0.9, beta2 0.999,
   eps 1e-8, step lr) on the mean of batch per-pair losses.  Loss of a pair: mean
   over its free DOFs of (y - target)^2.  *loss (optional): mean loss of the last epoch. */
WFFT_API int wfft_trainer_fit(wfft_trainer* t, int epochs, int batch, double lr, unsigned long long seed,
                              double* loss);
/* Current parameters as a model blob (bytes = wfft_model_bytes(hidden)). */
WFFT_API int wfft_trainer_get_model(const wfft_trainer* t, void* blob, size_t bytes);
WFFT_API const char* wfft_trainer_error(const wfft_trainer* t);
WFFT_API void wfft_trainer_destroy(wfft_trainer* t);

/* One evaluation of the network on a periodic grid n = {N1, N2, N3}: x is
   [V][16] FP32 host features (rounded to BF16 on the device), y receives
   [V][3] FP32 outputs. */
WFFT_API int wfft_net_forward(const void* blob, size_t bytes, const int n[3], const float* x, float* y);
/* Loss of one pair (mean over free DOFs of (y - target)^2, target [V][3], mask
   uint8 [V] with bit k set = component k prescribed, or NULL; c components) and its gradient
   w.r.t. the parameters (grad: FP32 in the blob's parameter layout). */
WFFT_API int wfft_net_loss_grad(const void* blob, size_t bytes, const int n[3], int c, const float* x,
                                const float* target, const unsigned char* mask, float* grad, double* loss);

/*
 * Autotuner (not in the paper).  Times, on this handle's grid and device, every
 * radix decomposition the FFT stages support for each axis (the power-of-two part
 * as radix-16 / radix-8 / radix-4 / one radix-2 stage in any mix), then the
 * x-pass tile size (1024, 2048, 4096 complex elements, capped by the register batch),
 * then every feasible column-tile width of each column pass, one choice at a time,
 * each candidate by
 * `reps` (0: 3) operator + preconditioner applications; keeps the fastest plan for
 * the handle's solve precision(s) and caches it per (precision, grid, device) for
 * later handles of the process (which then need no timing).  Plans that would need
 * more partial-sum slots than the handle allocated are skipped.  Only speed
 * changes: results may differ from the default plan in the last bits (a different
 * FFT rounding order), never beyond the solver tolerance.  *changed (optional):
 * how many choices differ from the handle's previous plan.  Overwrites the Krylov
 * scratch vectors (not the state); synchronises the stream; EINVAL while profiling.
 */
WFFT_API int wfft_autotune(wfft_handle* h, int reps, int* changed);
/*
 * Radix schedule of one axis of one precision's plan, set by hand: cnt[r] stages of
 * radix 8, 4, 2, 3, 5, 7, 16 (r = 0..6; their product, times the axis's prime factor
 * above 7 if it has one, must be the axis length).  The stages run in the order: the
 * prime factor's direct DFT stage (implied, not a choice), then 16s, 8s, 4s,
 * 2s, 3s, 5s, 7s.  The tile geometry follows; a schedule that would need more
 * partial-sum slots than the handle allocated is refused (EINVAL, plan unchanged).
 * Synchronises the stream.
 */
WFFT_API int wfft_set_radix(wfft_handle* h, int precision, int axis, const int cnt[7]);
/* The plan choices of one precision: radix[axis][r] stage counts (as wfft_set_radix),
   bx[axis][op] column-tile widths (axes 1, 2; op 0 forward, 1 inverse, 2 gradient, 3
   divergence, 4 preconditioner; powers of two up to 4, or 16 for the FP32 plain passes;
   256 | w with w = 4, 8 or 16 selects the register-stage kernels over a 256-point axis
   (FP32 3-D plans; tiles w columns wide); entries of passes the grid does not run are
   ignored) and
   xelems, the complex elements per x-pass tile (0 = the default 2048; 256..8192, capped
   by the register batch of the radix schedule); xelems | 65536 selects the
   register-stage x passes over 256-point rows (FP32 3-D plans, single-instance solves;
   at most 10 lines per tile of the 3-component passes and 5 of the middle pass).
   wfft_get_plan reads them (e.g. after wfft_autotune); wfft_set_plan applies them to a
   handle of the same grid, so a tuned plan can be kept and reused without timing.  A
   choice that does not fit the grid, the register batch, 64 KB of shared memory or the
   handle's partial-sum slots is refused (EINVAL, plan unchanged). */
typedef struct {
  int radix[3][7];
  int bx[3][5];
  int xelems;
} wfft_plan_choice;
WFFT_API int wfft_get_plan(const wfft_handle* h, int precision, wfft_plan_choice* out);
WFFT_API int wfft_set_plan(wfft_handle* h, int precision, const wfft_plan_choice* in);

/*
 * Explicit central-difference scheme (Sec. 2.3, Eq. Central_diff_rule, Eq.
 * Explicit_linear_momentum_arranged_3D), on a handle created with beta = 0,
 * gamma = 1/2.  One step, with the velocity Udot(t_n) prescribed on Gamma
 * (uniform per component, as U in wfft_step):
 *   u_n = u + dt v + dt^2/2 a on every DOF;
 *   v_b = v + dt/2 a + dt/(2 rho) div(C : grad^s u_n)   (the spectral operator, one FP64
 *         application, no Krylov solve);
 *   f_n = 2 rho/dt (Udot - v_b) on Gamma, 0 elsewhere;  v_n = v_b + dt/(2 rho) f_n (= Udot on Gamma);
 *   a_n = 2 (v_n - v)/dt - a.
 * info: iters 0, outer_applies 1, reaction = sum of f_n per component, ms.  The scheme is
 * conditionally stable: see wfft_explicit_dt.
 */
WFFT_API int wfft_explicit_step(wfft_handle* h, const double Udot[3], wfft_step_info* info);
/*
 * Largest stable increment of the explicit scheme (Eq. Courant_stable, Eq.
 * Eigenvalues_1D_homogeneo): 2 / omega_max, omega_max^2 the largest eigenvalue of
 * Q_ik = C_ijkl xi_j xi_l / rho at xi_i = N_i pi / L_i = pi / h_i, taken over the
 * nrows material rows (C: 21 Voigt values per row as in wfft_create, rho per row; 2-D
 * uses the in-plane block).  Host computation only (no GPU needed).  The operator's
 * own top frequency is below N_i pi / L_i (the Nyquist multiplier is 0), so this
 * bound is on the safe side.
 */
WFFT_API int wfft_explicit_dt(int ndim, const double h[3], const double* C, const double* rho, long long nrows,
                              double* dt_max);

/*
 * Upper bound of the largest eigenvalue of the operator A u = rho u + theta B^T C B u
 * (Eq. A_oper, Eq. G_oper) on the periodic grid n[] with voxel sizes h[]:
 * max rho + theta * max_x lambda_max(C(x)) * |xi|_max^2, lambda_max of C taken on
 * symmetric tensors (Mandel form of the Voigt matrix; 2-D: the in-plane block) and
 * |xi|_max^2 = sum_i (2 pi / (N_i h_i) * floor((N_i - 1) / 2))^2.  Exact per-row
 * eigenvalues up to 4096 rows, Gershgorin row sums above.  The incremental residual of
 * a mixed solve scales its rounding bound with this value.  Host computation only.
 */
WFFT_API int wfft_operator_bound(int ndim, const int n[3], const double h[3], const double* C, const double* rho,
                                 long long nrows, double theta, double* lam_max);

/*
 * Built-in FFT decomposition of an axis of n points (Sec. 2.1.3, Eq. Fourier_derivatives:
 * the DFT the transforms compute): cnt[r] stages of radix 8, 4, 2, 3, 5, 7, 16 (r = 0..6,
 * the layout of wfft_set_radix; the built-in schedule uses no radix-16 stage) and *prime =
 * the axis's prime factor above 7, taken by a direct prime-length DFT stage ahead of the
 * others (0: none).  This is the schedule a new handle starts from, unless the axis is
 * too long for the tiles of its passes (a handle then takes the decomposition whose
 * stages hold the most).  cnt and prime: caller-owned host arrays, written on success.
 * Returns WFFT_EINVAL (null pointers) or WFFT_EUNSUPPORTED (n outside 1..2048, two prime
 * factors above 7, or one above 127).  Host computation only.
 */
WFFT_API int wfft_axis_plan(int n, int cnt[7], int* prime);

/*
 * The paper's own treatment of the prescribed region (Sec. 2.2.3, Eqs. f_discrete,
 * solve_green, G, Vt, L-determination_ND; Alg. 2), for small regions; FP64 implicit
 * handles only.  wfft_green_setup solves A g = e_(p,j) without the projection P for a
 * unit force at every prescribed DOF (p, j) (PCG to tol), stores the responses at the
 * prescribed DOFs as column (p, j) of the dense Green's matrix G (row = responding
 * DOF), and inverts G on the GPU (Gauss-Jordan; G is symmetric positive definite).
 * It refuses more than max_dofs prescribed DOFs (0: 4096) -- G takes n^2 doubles and
 * n unit solves.  wfft_green_step then advances one Newmark step the paper's way:
 * u_b = A^-1 b (unconstrained, from u_{n-1}), V = U(t_n) - u_b on Gamma,
 * f = G^-1 V supported on Gamma, u_f = A^-1 f, u_n = u_b + u_f, then the corrector;
 * it gives the same u_n as wfft_step up to the solver tolerance.  info: iters of both
 * solves, outer_applies 2, reaction = sum rho a_n per component.
 */
WFFT_API int wfft_green_setup(wfft_handle* h, long long max_dofs);
WFFT_API int wfft_green_step(wfft_handle* h, const double U[3], wfft_step_info* info);

/* Kernel kinds of the launch accounting (wfft_profile_read). */
#define WFFT_K_XFWD_PLAIN 0   /* x-axis real->half-spectrum pass */
#define WFFT_K_XFWD_PUPD 1    /* ... fused with p = z + beta p */
#define WFFT_K_XFWD_RUPD 2    /* ... fused with x += alpha p, r -= alpha q, ||r||^2 */
#define WFFT_K_XFWD_CONV 3    /* ... fused with the FP64 -> FP32 residual conversion */
#define WFFT_K_XINV_APPLY 4   /* half-spectrum->real x pass fused with q = -theta t + rho p, mask, (p,q) */
#define WFFT_K_XINV_RESID 5   /* ... fused with r = P(b - A x), ||r||^2 (FP64) */
#define WFFT_K_XINV_PREC 6    /* ... fused with z = P(...) */
#define WFFT_K_XMID 7         /* x inverse + sigma = C(x):eps + x forward */
#define WFFT_K_COL_FWD 8      /* plain forward column (y / z) pass */
#define WFFT_K_COL_INV 9      /* plain inverse column pass */
#define WFFT_K_COL_GRAD 10    /* column pass fused with eps^ = sym(i xi (x) u^) */
#define WFFT_K_COL_DIV 11     /* column pass fused with t^ = i xi . sigma^ */
#define WFFT_K_COL_PREC 12    /* column pass fused with (theta K(xi) + rho_bar I)^-1 and Parseval (r,z) */
#define WFFT_K_NEWMARK 13     /* predictor / corrector */
#define WFFT_K_SCALAR 14      /* single-block finalize and bookkeeping kernels */
#define WFFT_K_NET_CONV 15    /* warm-start network convolutions (BF16 MMA, FP32 accumulate; counted as precision 1) */
#define WFFT_K_NET_AUX 16     /* warm-start scale, features, Taylor increment, training bookkeeping (precision 1) */
#define WFFT_K_XINV_PUPD 17   /* x inverse fused with z = P(...), p = z + beta p and the forward x transform of p */
#define WFFT_K_COUNT 18

/*
 * Launch accounting.  Every kernel launch of a handle is counted per kind and
 * precision.  wfft_profile(h, 1) resets the totals and brackets each
 * following launch with CUDA events on the handle's stream; wfft_profile(h, 0)
 * stops.  wfft_profile_read returns, for one (precision, kind): launches
 * counted, launches timed, their summed device time (ms), and their summed
 * algorithmic DRAM bytes and flops (the compulsory traffic / arithmetic of the
 * method, a model, not hardware counters).  Both synchronise the stream.
 */
WFFT_API int wfft_profile(wfft_handle* h, int enable);
WFFT_API int wfft_profile_read(wfft_handle* h, int precision, int kind, long long* launches, long long* timed,
                               double* ms, double* alg_bytes, double* alg_flops);
/* Total kernel launches issued by the handle since creation. */
WFFT_API int wfft_launch_count(const wfft_handle* h, long long* launches);

/*
 * Allocation-free preconditioner application: z = M r, FP64, unmasked -- the
 * same reference-medium preconditioner that wfft_precond applies -- for callers
 * that cannot allocate device memory: e.g. a framework that owns every device
 * byte through its own arena once it has started, or code that must not change
 * the device allocation state while other work is in flight.  It needs no
 * handle and performs no cudaMalloc / cudaFree or any other allocating call:
 * its scratch (kernel descriptor, scalars, twiddles, partial sums, spectral
 * work buffer) is one fixed __device__ array of 16.25 MiB in the library.  The
 * paper has no counterpart of this call.
 *   grid      : sizes as for wfft_create; c * N3 * N2 * pitch complex doubles must
 *               fit 16 MiB (pitch = N1/2+1 rounded up to 8), e.g. up to 64^3 in 3-D;
 *               larger grids return WFFT_EINVAL without touching the device.
 *   cbar      : 21 Voigt values of the reference stiffness (the volume average
 *               of C(x) for the paper's preconditioner); must be SPD.
 *   rho_bar   : reference density (> 0); theta = beta dt^2 (> 0).
 *   r_dev     : device FP64 [c][N3][N2][N1] input;  z_dev: device FP64 output;
 *               both must hold c * N1 * N2 * N3 doubles (the call cannot check this).
 *   stream    : cudaStream_t cast to void* (NULL = legacy default stream).
 * Asynchronous on `stream`.  Module loading: under CUDA's default lazy loading the
 * library's module, and with it the fixed array, is created on a device by the first
 * use of the library there (this call's first cudaGetSymbolAddress, or any earlier
 * launch of the library on that device); a caller whose arena will reserve all free
 * device memory should make a first call (or any other call of the library) before the
 * arena reserves it, or set CUDA_MODULE_LOADING=EAGER.  Every call looks up the array's
 * device address in the current context (cudaGetSymbolAddress, allocation-free once
 * the module is loaded); the first call in a CUDA context also sets the kernels'
 * shared-memory attributes, so make it before any stream capture.  All calls share
 * the one scratch array and it keeps the last call's contents: calls that overlap on
 * the GPU (other streams, other host threads) race and must be serialised by the
 * caller.  Errors: wfft_last_error(NULL) on the calling host thread.
 */
WFFT_API int wfft_precond_noalloc(const wfft_grid* grid, const double cbar[21], double rho_bar, double theta,
                                  const double* r_dev, double* z_dev, void* stream);

/* Query helpers. */
WFFT_API int wfft_get_sizes(const wfft_handle* h, int* ndim, int n[3], long long* nvox);
WFFT_API int wfft_device_bytes(const wfft_handle* h, size_t* bytes);

#ifdef __cplusplus
}
#endif
#endif /* WFFT_H */
