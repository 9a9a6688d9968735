// C ABI of libwfft (include/wfft.h): handle life cycle, host validation,
// FFT plans and twiddle tables, material and preconditioner tables, and the
// host orchestration of the preconditioned Krylov solve inside each
// beta-Newmark step (Alg. 2 loop body).  All arithmetic runs in the kernels
// of k_f64.cu / k_f32.cu; this file only allocates, uploads and launches.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/wfft.h"
#include "finalize.cuh"
#include "launch.cuh"
#include "passes.cuh"
#include "profiler.cuh"
#include "host_util.h"
#include "net.cuh"

using namespace wfft;

namespace wfft {
thread_local Profiler* g_prof = nullptr;
}

// Rounding constant of an FP32 operator application: ||fl32(A d) - A d|| is estimated
// as kIncrC u32 lam_max(A) ||d|| (u32 = 2^-24).  The ratio ||fl32(A d) - A d|| /
// (u32 lam_max ||d||) measures at most 0.7 on white noise (the worst input found) and
// about 0.2 on smooth fields, over 2-D / 3-D grids, phase and per-voxel tables and
// radix-16 plans; kIncrC is eleven times the largest, and the GPU tests require the
// measured ratio to stay below a quarter of it.
constexpr double kIncrC = 8.0;

struct wfft_handle {
  int ndim = 0, c = 0, s = 0;
  int n[3] = {1, 1, 1};
  double h[3] = {1, 1, 1};
  // 3-D grids with one voxel along x_1 run relabeled, (x_2, x_3, x_1) -> (x_1', x_2', x_3'):
  // internal component k is the caller's component cmap[k]; n_ext is the caller's grid
  bool relabeled = false;
  int cmap[3] = {0, 1, 2};
  int n_ext[3] = {1, 1, 1};
  long long V = 0;
  double dt = 0, beta = 0, gamma = 0, theta = 0;
  wfft_options opt{};
  cudaStream_t st = nullptr;
  Plan<double> P64;
  Plan<float> P32;
  Scalars* sc64 = nullptr;
  Scalars* sc32 = nullptr;
  Scalars* host_sc = nullptr;  // host-mapped pinned: [0] = sc64, [1] = sc32
  Scalars* host_sc_dev = nullptr;  // its device address
  std::vector<void*> dev_allocs;
  int nparts = 0;
  long long nstep = 0;
  bool has_mask = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  Profiler prof;
  bool au_valid = false;    // SL_AU holds A u for the current state u (mixed mode)
  bool last_resid_on_x = false;
  double lam_max = 0;       // upper bound of the largest eigenvalue of A (incremental residuals)
  double au_bound = 0;      // rounding estimate of SL_AU's latest update (0: full FP64)
  double U_prev[3] = {0, 0, 0};
  int gam_comp[3] = {0, 0, 0};  // 1: component j has prescribed DOFs (Gamma_j nonempty)
  double cbar[21] = {0};
  double rhobar = 0;
  // CUDA graphs of one block of check_every PCG iterations, per precision (captured lazily)
  cudaStream_t cap_st = nullptr;
  // asynchronous state downloads (wfft_download_async): copy stream, "state ready" and
  // "copies done" events; the next kernel that writes the state waits for the copies
  cudaStream_t dl_st = nullptr;
  cudaEvent_t dl_ready = nullptr, dl_done = nullptr;
  bool dl_pending = false;
  cudaGraphExec_t chunk[2] = {nullptr, nullptr};
  long long chunk_launches[2] = {0, 0};
  bool explicit_scheme = false;  // beta = 0, gamma = 1/2 (wfft_explicit_step)
  int solve_masked = 1;          // 0 while a Green's-matrix solve runs (no projection P)
  // Green's-matrix treatment of Gamma (wfft_green_setup)
  long long green_n = 0;         // prescribed DOFs
  long long* green_idx = nullptr;  // their global indices k V + vox, ascending
  double* green_ginv = nullptr;  // G^-1, row-major green_n x green_n
  double* green_v = nullptr;     // mismatch V
  double* green_f = nullptr;     // G^-1 V
  double* green_ub = nullptr;    // u_b of the current step
  double* green_piv = nullptr;
  NetDev* net = nullptr;    // learned warm start (wfft_set_model)
  NetWork nw;
  float* delta = nullptr;   // FP64 handles: FP32 warm-start increment
  std::string err;
};

// Makes the handle's profiler the current one for the launches of an API call.
struct ProfScope {
  Profiler* prev;
  explicit ProfScope(wfft_handle* h) : prev(g_prof) { g_prof = h ? &h->prof : nullptr; }
  ~ProfScope() { g_prof = prev; }
};

static thread_local std::string g_err;  // per host thread: calls without a handle may fail concurrently

namespace wfft {
// Error text of calls that have no handle (wfft_last_error(NULL)).
void set_global_error(const char* msg) { g_err = msg; }
}  // namespace wfft

static int fail(wfft_handle* h, int code, const std::string& msg) {
  if (h)
    h->err = msg;
  else
    g_err = msg;
  return code;
}

// Energy of the committed state (a sum over voxels, no cell volume):
// E_n = 1/2 sum rho |v_n|^2 + 1/2 sum eps_n : C : eps_n.  Implicit steps take the strain
// part from the step's own sums: the solve gives A u_n = b + theta f with f supported on
// Gamma, A = rho + theta K and u_n - u~ = theta a_n, so u.K u = -sum rho u_n . a_n +
// sum_j U_j F_j, where F_j = sum over Gamma_j of f_j equals the reaction sum rho a_n,j
// (the sum of K u over a periodic grid vanishes); exact up to the solver residual on the
// free DOFs.  Explicit steps have K u_n itself (esum = u_n . K u_n).
static double step_energy(const wfft_handle* h, const Scalars& s, const double U[3], bool explicit_step) {
  if (explicit_step) return 0.5 * s.ekin2 + 0.5 * s.esum;
  double w = -s.esum;
  for (int j = 0; j < 3; ++j)
    if (h->gam_comp[j]) w += U[j] * s.react[j];
  return 0.5 * s.ekin2 + 0.5 * w;
}

// Prescribed values in the handle's component order (the caller's U[cmap[k]]).
static void map_U(const wfft_handle* h, const double* U, double out[3]) {
  for (int k = 0; k < 3; ++k) out[k] = k < h->ndim ? U[h->cmap[k]] : 0.0;
}
// Reaction sums in the caller's component order.
static void put_reaction(const wfft_handle* h, const double* react, double out[3]) {
  for (int k = 0; k < 3; ++k) out[k] = 0.0;
  for (int k = 0; k < h->c; ++k) out[h->cmap[k]] = react[k];
}

#define CKH(h, x)                                                                                \
  do {                                                                                           \
    cudaError_t e_ = (x);                                                                        \
    if (e_ != cudaSuccess)                                                                       \
      return fail(h, WFFT_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_));               \
  } while (0)

template <typename P>
static cudaError_t dalloc(wfft_handle* h, P** ptr, size_t bytes) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess) return e;
  h->dev_allocs.push_back(p);
  *ptr = reinterpret_cast<P*>(p);
  return cudaSuccess;
}

template <typename T>
static int build_plan(wfft_handle* h, Plan<T>& P, const std::vector<double>& ctab21, int nrows,
                      const std::vector<double>& rhotab, const uint16_t* phase_dev, const uint8_t* mask_dev,
                      const double* cbar21, double rhobar) {
  Desc<T>& D = P.h;
  memset(&D, 0, sizeof(D));
  D.ndim = h->ndim;
  D.c = h->c;
  D.s = h->s;
  D.n1 = h->n[0];
  D.n2 = h->n[1];
  D.n3 = h->n[2];
  D.nh = D.n1 / 2 + 1;
  D.pitch = ((D.nh + 7) / 8) * 8;
  if (D.n3 > 1) {
    D.opAxis = 2;
    D.midAxis = D.n2 > 1 ? 1 : 0;
  } else {
    D.opAxis = 1;
    D.midAxis = 0;
  }
  D.V = h->V;
  D.Vh = (long long)D.n3 * D.n2 * D.pitch;
  const double twopi = 6.283185307179586476925286766559;
  D.kx1 = twopi / (h->n[0] * h->h[0]);
  D.kx2 = twopi / (h->n[1] * h->h[1]);
  D.kx3 = twopi / (h->n[2] * h->h[2]);
  D.ks[0] = (T)D.kx1;
  D.ks[1] = (T)D.kx2;
  D.ks[2] = (T)D.kx3;
  D.invV = (T)(1.0 / (double)h->V);
  D.theta = (T)h->theta;
  D.mthetaInvV = (T)(-h->theta / (double)h->V);
  D.rhobar = (T)rhobar;
  double kq[6][6];
  precond_coeffs(cbar21, h->theta, kq);
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) D.kq[a][b] = (T)kq[a][b];
  for (int ax = 0; ax < 3; ++ax) {
    if (!initial_schedule(h->n[ax], D.ax[ax], [](const AxisPlan& c) { return axis_tile_capacity<T>(c); }))
      return fail(h, WFFT_EUNSUPPORTED, "axis length not supported");
    // per-stage twiddles of the axis' radix schedule (rewritten by upload_desc when the
    // schedule changes)
    cplx<T>* dtw;
    CKH(h, dalloc(h, &dtw, (size_t)h->n[ax] * sizeof(cplx<T>)));
    D.tw[ax] = dtw;
  }
  // material tables in T
  const int stride = h->ndim == 3 ? kCtabStride3 : kCtabStride2;
  std::vector<T> ct((size_t)nrows * stride, (T)0);
  const int idx2[6] = {0, 1, 5, 6, 10, 20};
  for (int r = 0; r < nrows; ++r) {
    if (h->ndim == 3)
      for (int k = 0; k < 21; ++k) ct[(size_t)r * stride + k] = (T)ctab21[(size_t)r * 21 + k];
    else
      for (int k = 0; k < 6; ++k) ct[(size_t)r * stride + k] = (T)ctab21[(size_t)r * 21 + idx2[k]];
  }
  T* dct;
  CKH(h, dalloc(h, &dct, ct.size() * sizeof(T)));
  CKH(h, cudaMemcpy(dct, ct.data(), ct.size() * sizeof(T), cudaMemcpyHostToDevice));
  D.ctab = dct;
  std::vector<T> rt(rhotab.size());
  for (size_t i = 0; i < rt.size(); ++i) rt[i] = (T)rhotab[i];
  T* drt;
  CKH(h, dalloc(h, &drt, rt.size() * sizeof(T)));
  CKH(h, cudaMemcpy(drt, rt.data(), rt.size() * sizeof(T), cudaMemcpyHostToDevice));
  D.rhotab = drt;
  D.phase = phase_dev;
  D.mask = mask_dev;
  D.dt = h->dt;
  D.beta = h->beta;
  D.gamma = h->gamma;
  plan_geometry<T>(P);
  if (!P.g.fits)
    return fail(h, WFFT_EUNSUPPORTED, "an axis is too long for the passes' tiles (register batch or shared memory)");
  // spectral buffer and Krylov vectors in T
  cplx<T>* spec;
  CKH(h, dalloc(h, &spec, (size_t)D.s * D.Vh * sizeof(cplx<T>)));
  // the pitch padding of the rows is never written by the passes: zero it once, so that
  // copies of whole rows (wfft_rfft3) carry zeros there
  CKH(h, cudaMemset(spec, 0, (size_t)D.s * D.Vh * sizeof(cplx<T>)));
  D.spec = spec;
  const size_t vec = (size_t)h->c * h->V;
  for (int sl : {(int)SL_R, (int)SL_Z, (int)SL_P, (int)SL_Q}) {
    T* p;
    CKH(h, dalloc(h, &p, vec * sizeof(T)));
    CKH(h, cudaMemset(p, 0, vec * sizeof(T)));
    D.slot[sl] = p;
  }
  return WFFT_OK;
}

// Descriptor and the per-stage twiddle tables of its radix schedules to the device.
template <typename T>
static cudaError_t upload_desc(Plan<T>& P) {
  if (!P.d) {
    cudaError_t e = cudaMalloc(&P.d, sizeof(Desc<T>));
    if (e != cudaSuccess) return e;
  }
  for (int ax = 0; ax < 3; ++ax) {
    std::vector<cplx<T>> w((size_t)P.h.ax[ax].n);
    fill_stage_twiddles<T>(w.data(), P.h.ax[ax]);
    cudaError_t e = cudaMemcpy(const_cast<cplx<T>*>(P.h.tw[ax]), w.data(), w.size() * sizeof(cplx<T>),
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  return cudaMemcpy(P.d, &P.h, sizeof(Desc<T>), cudaMemcpyHostToDevice);
}

template <typename T>
static cudaError_t set_ext(Plan<T>& P, const void* in, void* out, cudaStream_t st) {
  P.h.slot[SL_EXT_IN] = const_cast<void*>(in);
  P.h.slot[SL_EXT_OUT] = out;
  return cudaMemcpyAsync(&P.d->slot[SL_EXT_IN], &P.h.slot[SL_EXT_IN], 2 * sizeof(void*), cudaMemcpyHostToDevice,
                         st);
}

extern "C" int wfft_default_options(wfft_options* o) {
  if (!o) return WFFT_EINVAL;
  o->precision = WFFT_FP64;
  o->tol = 1e-10;
  o->maxit = 1000;
  o->warm_start = WFFT_WARM_PREV;
  o->inner_tol = 1e-5;
  o->max_sweeps = 20;
  o->check_every = 4;
  o->use_graphs = 1;
  o->inner_floor = 0.5;
  o->incr_resid = 1;
  o->watchdog_iters = 0;
  return WFFT_OK;
}

static int init_attrs_once(wfft_handle* h) {
  static int done = 0;
  if (done) return WFFT_OK;
  CKH(h, init_kernel_attributes<double>());
  CKH(h, init_kernel_attributes<float>());
  done = 1;
  return WFFT_OK;
}

extern "C" int wfft_create(const wfft_grid* grid, const double* C, const uint16_t* phase, int nphase,
                           const double* rho, const uint8_t* mask, double dt, double beta, double gamma,
                           const wfft_options* opt, void* stream, wfft_handle** out) {
  if (!out) return fail(nullptr, WFFT_EINVAL, "out is NULL");
  *out = nullptr;
  if (!grid || !C || !rho) return fail(nullptr, WFFT_EINVAL, "grid, C and rho are required");
  if (grid->ndim != 2 && grid->ndim != 3) return fail(nullptr, WFFT_EINVAL, "ndim must be 2 or 3");
  for (int i = 0; i < 3; ++i) {
    if (grid->n[i] < 1) return fail(nullptr, WFFT_EINVAL, "grid sizes must be >= 1");
    if (!(grid->h[i] > 0)) return fail(nullptr, WFFT_EINVAL, "voxel sizes must be > 0");
  }
  if (grid->ndim == 2 && grid->n[2] != 1) return fail(nullptr, WFFT_EINVAL, "2-D grids need n[2] == 1");
  if (grid->n[1] == 1 && grid->n[2] == 1) return fail(nullptr, WFFT_EUNSUPPORTED, "N2 = N3 = 1 is not supported");
  if (grid->ndim == 3 && grid->n[0] == 1) {
    // One voxel along x_1 (the paper's 1 x N x N plates, Sec. 4.1): run the same medium on
    // the cyclically relabeled axes (x_1', x_2', x_3') = (x_2, x_3, x_1), grid (N2, N3, 1).
    // With N1 = 1 the voxel order [N3][N2][1] is [1][N3][N2]: voxel arrays are unchanged;
    // component k' is the caller's component cmap[k'] = (1, 2, 0)[k'], and the stiffness is
    // relabeled index by index (Voigt 11 <- 22, 22 <- 33, 33 <- 11, 23 <- 13, 13 <- 12, 12 <- 23).
    if (grid->n[2] == 1) return fail(nullptr, WFFT_EUNSUPPORTED, "N1 = N3 = 1 is not supported");
    const long long Vx = (long long)grid->n[1] * grid->n[2];
    const int cm[3] = {1, 2, 0};
    const int vm[6] = {1, 2, 0, 4, 5, 3};
    const long long rows = phase ? (nphase > 0 ? nphase : 0) : Vx;
    std::vector<double> C2((size_t)rows * 21);
    for (long long r = 0; r < rows; ++r) {
      double m6[36], m2[36];
      voigt_full(C + (size_t)r * 21, m6);
      for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) m2[a * 6 + b] = m6[vm[a] * 6 + vm[b]];
      int k = 0;
      for (int a = 0; a < 6; ++a)
        for (int b = a; b < 6; ++b) C2[(size_t)r * 21 + k++] = m2[a * 6 + b];
    }
    std::vector<uint8_t> M2;
    if (mask) {
      M2.resize((size_t)3 * Vx);
      for (int k = 0; k < 3; ++k) memcpy(&M2[(size_t)k * Vx], mask + (size_t)cm[k] * Vx, (size_t)Vx);
    }
    wfft_grid g2;
    g2.ndim = 3;
    g2.n[0] = grid->n[1];
    g2.n[1] = grid->n[2];
    g2.n[2] = 1;
    g2.h[0] = grid->h[1];
    g2.h[1] = grid->h[2];
    g2.h[2] = grid->h[0];
    const int rc = wfft_create(&g2, C2.data(), phase, nphase, rho, mask ? M2.data() : nullptr, dt, beta, gamma,
                               opt, stream, out);
    if (rc == WFFT_OK) {
      wfft_handle* hr = *out;
      hr->relabeled = true;
      for (int k = 0; k < 3; ++k) {
        hr->cmap[k] = cm[k];
        hr->n_ext[k] = grid->n[k];
      }
    }
    return rc;
  }
  const bool explicit_scheme = beta == 0.0 && gamma == 0.5;
  if (!(dt > 0) || !(gamma >= 0) || !(beta > 0 || explicit_scheme))
    return fail(nullptr, WFFT_EINVAL, "need dt > 0, gamma >= 0 and beta > 0 (or beta = 0, gamma = 1/2: explicit scheme)");
  if (explicit_scheme && opt && opt->precision != WFFT_FP64)
    return fail(nullptr, WFFT_EINVAL, "the explicit scheme runs in FP64");
  if (phase && nphase < 1) return fail(nullptr, WFFT_EINVAL, "nphase must be >= 1");
  for (int i = 0; i < 3; ++i) {
    AxisPlan pl;
    if (!factorize(grid->n[i], pl))
      return fail(nullptr, WFFT_EUNSUPPORTED,
                  "axis lengths must have prime factors 2, 3, 5, 7 and at most one other prime, up to 127");
  }
  wfft_handle* h = new (std::nothrow) wfft_handle();
  if (!h) return fail(nullptr, WFFT_ENOMEM, "host allocation failed");
  h->ndim = grid->ndim;
  h->c = grid->ndim;
  h->s = grid->ndim == 3 ? 6 : 3;
  for (int i = 0; i < 3; ++i) {
    h->n[i] = grid->n[i];
    h->n_ext[i] = grid->n[i];
    h->h[i] = grid->h[i];
  }
  h->V = (long long)grid->n[0] * grid->n[1] * grid->n[2];
  h->dt = dt;
  h->beta = beta;
  h->gamma = gamma;
  // the explicit scheme has no solve: its operator passes run at theta = 1, so the
  // divergence pass returns -div(C : grad^s u) itself
  h->explicit_scheme = explicit_scheme;
  h->theta = explicit_scheme ? 1.0 : beta * dt * dt;
  if (opt)
    h->opt = *opt;
  else
    wfft_default_options(&h->opt);
  if (h->opt.check_every < 1) h->opt.check_every = 1;
  if (h->opt.maxit < 1) h->opt.maxit = 1000;
  if (h->opt.max_sweeps < 1) h->opt.max_sweeps = 20;
  if (!(h->opt.inner_tol > 0)) h->opt.inner_tol = 1e-4;
  if (h->opt.precision != WFFT_FP64 && h->opt.precision != WFFT_MIXED) {
    delete h;
    return fail(nullptr, WFFT_EINVAL, "unknown precision");
  }
  h->st = reinterpret_cast<cudaStream_t>(stream);
  // ---- validate and reduce the material on the host
  const long long V = h->V;
  const int nrows = phase ? nphase : (int)std::min<long long>(V, 0x7fffffff);
  if (!phase && V > 0x7fffffffLL) {
    delete h;
    return fail(nullptr, WFFT_EINVAL, "grid too large for per-voxel tables");
  }
  std::vector<double> ctab(C, C + (size_t)nrows * 21), rtab(rho, rho + nrows);
  for (int r = 0; r < nrows; ++r) {
    if (!(rtab[r] > 0)) {
      delete h;
      return fail(nullptr, WFFT_EINVAL, "rho must be > 0");
    }
    double m6[36];
    voigt_full(&ctab[(size_t)r * 21], m6);
    bool ok;
    if (h->ndim == 3) {
      ok = spd(m6, 6);
    } else {
      const int id[3] = {0, 1, 5};
      double m3[9];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) m3[a * 3 + b] = m6[id[a] * 6 + id[b]];
      ok = spd(m3, 3);
    }
    if (!ok) {
      delete h;
      return fail(nullptr, WFFT_EINVAL, "stiffness is not symmetric positive definite");
    }
  }
  std::vector<double> counts(nrows, 0.0);
  if (phase) {
    for (long long v = 0; v < V; ++v) {
      if (phase[v] >= nphase) {
        delete h;
        return fail(nullptr, WFFT_EINVAL, "phase id out of range");
      }
      counts[phase[v]] += 1.0;
    }
  } else {
    for (int r = 0; r < nrows; ++r) counts[r] = 1.0;
  }
  double cbar[21] = {0}, rhobar = 0;
  for (int r = 0; r < nrows; ++r) {
    if (counts[r] == 0) continue;
    for (int k = 0; k < 21; ++k) cbar[k] += counts[r] * ctab[(size_t)r * 21 + k];
    rhobar += counts[r] * rtab[r];
  }
  for (int k = 0; k < 21; ++k) cbar[k] /= (double)V;
  rhobar /= (double)V;
  for (int k = 0; k < 21; ++k) h->cbar[k] = cbar[k];
  h->rhobar = rhobar;
  h->lam_max = explicit_scheme ? 0.0 : operator_max_eig_bound(h->ndim, h->n, h->h, ctab.data(), rtab.data(), nrows,
                                                              h->theta);
  // per-voxel component mask bits
  std::vector<uint8_t> mbits((size_t)V, 0);
  long long nfixed = 0;
  if (mask) {
    for (int k = 0; k < h->c; ++k)
      for (long long v = 0; v < V; ++v)
        if (mask[(size_t)k * V + v]) {
          mbits[v] |= (uint8_t)(1u << k);
          ++nfixed;
        }
  }
  h->has_mask = nfixed > 0;
  for (int k = 0; k < h->c; ++k) {
    const uint8_t bit = (uint8_t)(1u << k);
    for (long long v = 0; v < V && !h->gam_comp[k]; ++v)
      if (mbits[v] & bit) h->gam_comp[k] = 1;
  }
  if (nfixed >= (long long)h->c * V) {
    delete h;
    return fail(nullptr, WFFT_EINVAL, "the mask covers every DOF");
  }
  // ---- device uploads (every host-side check has passed)
  int rc = init_attrs_once(h);
  if (rc) {
    std::string m = h->err;
    delete h;
    return fail(nullptr, rc, m);
  }
  uint16_t* dphase = nullptr;
  uint8_t* dmask = nullptr;
#define CKC(x)                                                 \
  do {                                                         \
    cudaError_t e_ = (x);                                      \
    if (e_ != cudaSuccess) {                                   \
      std::string m_ = std::string(#x) + ": " + cudaGetErrorString(e_); \
      wfft_destroy(h);                                         \
      return fail(nullptr, WFFT_ECUDA, m_);                    \
    }                                                          \
  } while (0)
  if (phase) {
    CKC(dalloc(h, &dphase, (size_t)V * sizeof(uint16_t)));
    CKC(cudaMemcpy(dphase, phase, (size_t)V * sizeof(uint16_t), cudaMemcpyHostToDevice));
  }
  CKC(dalloc(h, &dmask, (size_t)V));
  CKC(cudaMemcpy(dmask, mbits.data(), (size_t)V, cudaMemcpyHostToDevice));
  rc = build_plan<double>(h, h->P64, ctab, nrows, rtab, dphase, dmask, cbar, rhobar);
  if (rc == WFFT_OK) rc = build_plan<float>(h, h->P32, ctab, nrows, rtab, dphase, dmask, cbar, rhobar);
  if (rc != WFFT_OK) {
    std::string m = h->err;
    wfft_destroy(h);
    return fail(nullptr, rc, m);
  }
  // FP64 state, rhs, solution, FP64 residual, lifting fields
  const size_t vec = (size_t)h->c * V;
  Desc<double>& D = h->P64.h;
  for (int sl : {(int)SL_U, (int)SL_V, (int)SL_A, (int)SL_B, (int)SL_X, (int)SL_R64}) {
    double* p;
    CKC(dalloc(h, &p, vec * sizeof(double)));
    CKC(cudaMemset(p, 0, vec * sizeof(double)));
    D.slot[sl] = p;
  }
  if (h->opt.precision == WFFT_FP64) {
    D.slot[SL_R64] = D.slot[SL_R];
  } else {
    double* au;
    CKC(dalloc(h, &au, vec * sizeof(double)));
    CKC(cudaMemset(au, 0, vec * sizeof(double)));
    D.slot[SL_AU] = au;
  }
  double* w;
  CKC(dalloc(h, &w, vec * h->ndim * sizeof(double)));
  CKC(cudaMemset(w, 0, vec * h->ndim * sizeof(double)));
  D.slot[SL_W] = w;
  // the FP32 plan shares the FP64 state / solution / residual / lifting slots
  Desc<float>& F = h->P32.h;
  for (int sl : {(int)SL_U, (int)SL_V, (int)SL_A, (int)SL_B, (int)SL_X, (int)SL_W}) F.slot[sl] = D.slot[sl];
  F.slot[SL_R64] = h->opt.precision == WFFT_FP64 ? nullptr : D.slot[SL_R64];
  if (h->opt.precision == WFFT_MIXED) {
    // FP32 correction of the inner solve, folded into x by the FP64 residual pass
    float* dcor;
    CKC(dalloc(h, &dcor, vec * sizeof(float)));
    CKC(cudaMemset(dcor, 0, vec * sizeof(float)));
    F.slot[SL_D] = dcor;
    D.slot[SL_D] = dcor;
  }
  // partial sums and scalars
  // room for the block partial sums of any column-tile width (grouped launches may
  // use a narrower tile than the instance's own plan)
  const int colmax = (h->n[0] / 2 + 1) * std::max(h->n[1], h->n[2]);
  h->nparts = std::max({h->P64.g.max_blocks, h->P32.g.max_blocks, kEwBlocks, colmax});
  for (int k = 0; k < NPART; ++k) {
    CKC(dalloc(h, &D.part[k], (size_t)h->nparts * sizeof(double)));
    CKC(dalloc(h, &F.part[k], (size_t)h->nparts * sizeof(double)));
  }
  CKC(dalloc(h, &h->sc64, sizeof(Scalars)));
  CKC(dalloc(h, &h->sc32, sizeof(Scalars)));
  CKC(cudaMemset(h->sc64, 0, sizeof(Scalars)));
  CKC(cudaMemset(h->sc32, 0, sizeof(Scalars)));
  D.sc = h->sc64;
  F.sc = h->sc32;
  D.sc_inner = h->sc32;
  CKC(cudaHostAlloc(&h->host_sc, 2 * sizeof(Scalars), cudaHostAllocMapped));
  CKC(cudaHostGetDevicePointer(reinterpret_cast<void**>(&h->host_sc_dev), h->host_sc, 0));
  memset(h->host_sc, 0, 2 * sizeof(Scalars));
  CKC(upload_desc(h->P64));
  CKC(upload_desc(h->P32));
  CKC(cudaEventCreate(&h->ev0));
  CKC(cudaEventCreate(&h->ev1));
  // lifting fields w_j = P A(E e_j) for the stopping-test reference norm
  ProfScope ps_(h);
  if (h->has_mask && !h->explicit_scheme) {
    double* tmp = reinterpret_cast<double*>(D.slot[SL_Z]);
    for (int j = 0; j < h->ndim; ++j) {
      launch_set_done(h->sc64, 0, h->st);
      launch_fill_unit(h->P64, j, tmp, h->st);
      CKC(set_ext(h->P64, tmp, w + (size_t)j * vec, h->st));
      launch_apply<double>(h->P64, PRE_PLAIN, SL_EXT_IN, POST_APPLY, SL_EXT_OUT, 1, 0, h->st);
    }
  }
  CKC(cudaGetLastError());
  CKC(cudaStreamSynchronize(h->st));
#undef CKC
  *out = h;
  return WFFT_OK;
}

extern "C" void wfft_destroy(wfft_handle* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  for (int k = 0; k < 2; ++k)
    if (h->chunk[k]) cudaGraphExecDestroy(h->chunk[k]);
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  if (h->dl_st) {
    cudaStreamSynchronize(h->dl_st);
    cudaStreamDestroy(h->dl_st);
  }
  if (h->dl_ready) cudaEventDestroy(h->dl_ready);
  if (h->dl_done) cudaEventDestroy(h->dl_done);
  for (void* p : h->dev_allocs) cudaFree(p);
  net_free(h->net);
  net_work_free(&h->nw);
  if (h->P64.d) cudaFree(h->P64.d);
  if (h->P32.d) cudaFree(h->P32.d);
  if (h->host_sc) cudaFreeHost(h->host_sc);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  delete h;
}

extern "C" const char* wfft_last_error(const wfft_handle* h) { return h ? h->err.c_str() : g_err.c_str(); }

extern "C" int wfft_get_sizes(const wfft_handle* h, int* ndim, int n[3], long long* nvox) {
  if (!h) return WFFT_EINVAL;
  if (ndim) *ndim = h->ndim;
  if (n)
    for (int i = 0; i < 3; ++i) n[i] = h->n_ext[i];
  if (nvox) *nvox = h->V;
  return WFFT_OK;
}

extern "C" int wfft_device_bytes(const wfft_handle* h, size_t* bytes) {
  if (!h || !bytes) return WFFT_EINVAL;
  const size_t vec = (size_t)h->c * h->V;
  const Desc<double>& D = h->P64.h;
  size_t b = vec * 8 * (6 + h->ndim) + vec * (8 + 4) * 4 + (size_t)h->s * D.Vh * (16 + 8) + (size_t)h->V * 3;
  *bytes = b;
  return WFFT_OK;
}

extern "C" int wfft_spectral_pitch(const wfft_handle* h, int* pitch) {
  if (!h || !pitch) return WFFT_EINVAL;
  *pitch = h->P64.h.pitch;
  return WFFT_OK;
}

// Orders the next state write on stream st after the pending asynchronous downloads.
static int wait_downloads(wfft_handle* h, cudaStream_t st) {
  if (!h->dl_pending) return WFFT_OK;
  CKH(h, cudaStreamWaitEvent(st, h->dl_done, 0));
  if (st == h->st) h->dl_pending = false;
  return WFFT_OK;
}

static int state_copy(wfft_handle* h, int to_dev, double* u, double* v, double* a, cudaMemcpyKind kind) {
  const size_t bytes = (size_t)h->c * h->V * sizeof(double);
  if (to_dev) {
    int rc = wait_downloads(h, h->st);
    if (rc) return rc;
  }
  double* dst[3] = {(double*)h->P64.h.slot[SL_U], (double*)h->P64.h.slot[SL_V], (double*)h->P64.h.slot[SL_A]};
  double* src[3] = {u, v, a};
  const size_t cb = (size_t)h->V * sizeof(double);  // one component
  for (int i = 0; i < 3; ++i) {
    if (to_dev) {
      if (!src[i]) {
        CKH(h, cudaMemsetAsync(dst[i], 0, bytes, h->st));
      } else if (!h->relabeled) {
        CKH(h, cudaMemcpyAsync(dst[i], src[i], bytes, kind, h->st));
      } else {
        for (int k = 0; k < h->c; ++k)
          CKH(h, cudaMemcpyAsync(dst[i] + (size_t)k * h->V, src[i] + (size_t)h->cmap[k] * h->V, cb, kind, h->st));
      }
    } else if (src[i]) {
      if (!h->relabeled) {
        CKH(h, cudaMemcpyAsync(src[i], dst[i], bytes, kind, h->st));
      } else {
        for (int k = 0; k < h->c; ++k)
          CKH(h, cudaMemcpyAsync(src[i] + (size_t)h->cmap[k] * h->V, dst[i] + (size_t)k * h->V, cb, kind, h->st));
      }
    }
  }
  CKH(h, cudaStreamSynchronize(h->st));
  return WFFT_OK;
}

extern "C" int wfft_download_async(wfft_handle* h, double* u, double* v, double* a) {
  if (!h) return fail(nullptr, WFFT_EINVAL, "null handle");
  if (!h->dl_st) {
    CKH(h, cudaStreamCreateWithFlags(&h->dl_st, cudaStreamNonBlocking));
    CKH(h, cudaEventCreateWithFlags(&h->dl_ready, cudaEventDisableTiming));
    CKH(h, cudaEventCreateWithFlags(&h->dl_done, cudaEventDisableTiming));
  }
  const size_t bytes = (size_t)h->c * h->V * sizeof(double);
  double* src[3] = {(double*)h->P64.h.slot[SL_U], (double*)h->P64.h.slot[SL_V], (double*)h->P64.h.slot[SL_A]};
  double* dst[3] = {u, v, a};
  CKH(h, cudaEventRecord(h->dl_ready, h->st));
  CKH(h, cudaStreamWaitEvent(h->dl_st, h->dl_ready, 0));
  for (int i = 0; i < 3; ++i) {
    if (!dst[i]) continue;
    if (!h->relabeled) {
      CKH(h, cudaMemcpyAsync(dst[i], src[i], bytes, cudaMemcpyDeviceToHost, h->dl_st));
    } else {
      const size_t cb = (size_t)h->V * sizeof(double);
      for (int k = 0; k < h->c; ++k)
        CKH(h, cudaMemcpyAsync(dst[i] + (size_t)h->cmap[k] * h->V, src[i] + (size_t)k * h->V, cb,
                               cudaMemcpyDeviceToHost, h->dl_st));
    }
  }
  CKH(h, cudaEventRecord(h->dl_done, h->dl_st));
  h->dl_pending = true;
  return WFFT_OK;
}

extern "C" int wfft_download_wait(wfft_handle* h) {
  if (!h) return fail(nullptr, WFFT_EINVAL, "null handle");
  if (h->dl_done) CKH(h, cudaEventSynchronize(h->dl_done));
  return WFFT_OK;
}

extern "C" int wfft_set_state(wfft_handle* h, const double* u, const double* v, const double* a, long long n) {
  if (!h) return fail(nullptr, WFFT_EINVAL, "null handle");
  h->nstep = n;
  h->au_valid = false;
  return state_copy(h, 1, (double*)u, (double*)v, (double*)a, cudaMemcpyHostToDevice);
}
extern "C" int wfft_get_state(const wfft_handle* hc, double* u, double* v, double* a, long long* n) {
  wfft_handle* h = const_cast<wfft_handle*>(hc);
  if (!h) return fail(nullptr, WFFT_EINVAL, "null handle");
  if (n) *n = h->nstep;
  return state_copy(h, 0, u, v, a, cudaMemcpyDeviceToHost);
}
extern "C" int wfft_set_state_dev(wfft_handle* h, const double* u, const double* v, const double* a, long long n) {
  if (!h) return fail(nullptr, WFFT_EINVAL, "null handle");
  h->nstep = n;
  h->au_valid = false;
  return state_copy(h, 1, (double*)u, (double*)v, (double*)a, cudaMemcpyDeviceToDevice);
}
extern "C" int wfft_get_state_dev(const wfft_handle* hc, double* u, double* v, double* a) {
  wfft_handle* h = const_cast<wfft_handle*>(hc);
  if (!h) return fail(nullptr, WFFT_EINVAL, "null handle");
  return state_copy(h, 0, u, v, a, cudaMemcpyDeviceToDevice);
}

// Host field [c][V] of the caller <-> device field of the handle (component order cmap).
static int field_copy(wfft_handle* h, void* dst, const void* src, cudaMemcpyKind kind) {
  const size_t cb = (size_t)h->V * sizeof(double);
  if (!h->relabeled) {
    CKH(h, cudaMemcpyAsync(dst, src, cb * h->c, kind, h->st));
    return WFFT_OK;
  }
  const bool to_dev = kind == cudaMemcpyHostToDevice;
  for (int k = 0; k < h->c; ++k) {
    const size_t di = (size_t)(to_dev ? k : h->cmap[k]) * cb, si = (size_t)(to_dev ? h->cmap[k] : k) * cb;
    CKH(h, cudaMemcpyAsync((char*)dst + di, (const char*)src + si, cb, kind, h->st));
  }
  return WFFT_OK;
}

static int read_scalars(wfft_handle* h) {
  launch_read_scalars(h->sc64, h->sc32, h->host_sc_dev, h->st);
  CKH(h, cudaGetLastError());
  CKH(h, cudaStreamSynchronize(h->st));
  return WFFT_OK;
}

// One block of check_every PCG iterations on stream st (every kernel returns at once
// when the solve's done flag is set, so a block may overrun convergence harmlessly).
template <typename T>
static void pcg_chunk(wfft_handle* h, Plan<T>& P, Scalars* sc, cudaStream_t st, int count) {
  const Desc<T>& D = P.h;
  const int op = D.opAxis;
  const int m = h->solve_masked;
  for (int i = 0; i < count; ++i) {
    // q = P A p from the half spectrum of p left by the previous preconditioner pass
    launch_apply<T>(P, PRE_NONE, SL_P, POST_APPLY, SL_Q, m, 1, st);
    launch_fin(sc, D.part[PT_A], P.g.blk_x, nullptr, 0, nullptr, 0, FIN_ALPHA, nullptr, st);
    // x += alpha p, r -= alpha q, ||r||^2, M r up to the Parseval (r, z); beta; then
    // z, p = z + beta p and the half spectrum of p
    launch_precond_part_impl<T>(P, 0, PRE_RUPD, SL_R, m, st);
    launch_fin(sc, D.part[PT_A], P.g.blk_x, D.part[PT_B], P.g.blk_col[op][OP_PREC], nullptr, 0, FIN_BETA, nullptr, st);
    launch_precond_part_impl<T>(P, 1, 0, 0, m, st);
  }
}

// First preconditioner application of a solve (or of a mixed inner solve): z = M r
// with the x-pass prologue `pre`, (r, z), and the first search direction p = z with
// its half spectrum.
template <typename T>
static void precond_start(Plan<T>& P, Scalars* sc, int pre, int masked, cudaStream_t st) {
  const Desc<T>& D = P.h;
  launch_precond_part_impl<T>(P, 0, pre, SL_R, masked, st);
  launch_fin(sc, nullptr, 0, D.part[PT_B], P.g.blk_col[D.opAxis][OP_PREC], nullptr, 0, FIN_RZ0, nullptr, st);
  launch_precond_part_impl<T>(P, 1, 0, 0, masked, st);
}

// Launch one block of iterations, as a CUDA graph when enabled: the block is captured
// once per handle and precision on the handle's internal stream (capture needs a
// stream other than the legacy default one) and replayed on the solve's stream.
// Every kernel argument is a pointer to device-resident descriptors and scalars,
// so a replay computes exactly what direct launches would.
// While profiling, blocks are one iteration long: the iterations of a block that follow
// convergence launch kernels that return at once, and those would bias the per-launch
// times of the kernel table.
template <typename T>
static int chunk_len(const wfft_handle* h) {
  return h->prof.on ? 1 : h->opt.check_every;
}

template <typename T>
static int pcg_chunk_launch(wfft_handle* h, Plan<T>& P, Scalars* sc, int which) {
  if (!h->opt.use_graphs || h->prof.on || !h->solve_masked) {
    pcg_chunk<T>(h, P, sc, h->st, chunk_len<T>(h));
    return WFFT_OK;
  }
  if (!h->chunk[which]) {
    if (!h->cap_st) CKH(h, cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
    const long long before = h->prof.lifetime;
    cudaGraph_t g = nullptr;
    CKH(h, cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal));
    pcg_chunk<T>(h, P, sc, h->cap_st, h->opt.check_every);
    const cudaError_t ec = cudaStreamEndCapture(h->cap_st, &g);
    if (ec != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      return fail(h, WFFT_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
    }
    const cudaError_t ei = cudaGraphInstantiate(&h->chunk[which], g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      h->chunk[which] = nullptr;
      return fail(h, WFFT_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
    }
    // the capture counted the block's kernels once; they are counted again per replay
    h->chunk_launches[which] = h->prof.lifetime - before;
    h->prof.lifetime = before;
  }
  CKH(h, cudaGraphLaunch(h->chunk[which], h->st));
  h->prof.lifetime += h->chunk_launches[which];
  return WFFT_OK;
}

// PCG iterations on plan P (scalars sc) until its done flag is set; counts in *iters.
template <typename T>
static int pcg_loop(wfft_handle* h, Plan<T>& P, Scalars* sc, int which, int budget, int* iters) {
  int launched = 0;
  for (;;) {
    const int len = chunk_len<T>(h);
    int rc0 = pcg_chunk_launch<T>(h, P, sc, which);
    if (rc0) return rc0;
    launched += len;
    CKH(h, cudaGetLastError());
    int rc = read_scalars(h);
    if (rc) return rc;
    const Scalars& s = h->host_sc[which];
    if (s.done) {
      *iters = s.iter;
      return WFFT_OK;
    }
    if (launched >= budget) {
      *iters = s.iter;
      return WFFT_ETIMEOUT;
    }
  }
}

// Solve with B, X set and sc64->ref2 known; fills status / counts.
static int solve_core(wfft_handle* h, wfft_step_info* info, bool use_au = false, bool inner_guess = false) {
  Plan<double>& P = h->P64;
  const Desc<double>& D = P.h;
  const int watchdog = h->opt.watchdog_iters > 0 ? h->opt.watchdog_iters : 4 * h->opt.maxit;
  int iters = 0, outer = 0, sweeps = 0, incr_count = 0;
  int status = WFFT_OK;
  if (h->opt.precision == WFFT_FP64) {
    launch_apply<double>(P, PRE_PLAIN, SL_X, POST_RESID, 0, 1, 1, h->st);
    launch_fin(h->sc64, D.part[PT_A], P.g.blk_x, nullptr, 0, nullptr, 0, FIN_RES0, nullptr, h->st);
    precond_start<double>(P, h->sc64, PRE_PLAIN, 1, h->st);
    outer = 1;
    int rc = pcg_loop<double>(h, P, h->sc64, 0, watchdog, &iters);
    if (rc == WFFT_ETIMEOUT) status = WFFT_ETIMEOUT;
    else if (rc) return rc;
    if (!status) status = h->host_sc[0].status;
  } else {
    Plan<float>& F = h->P32;
    const Desc<float>& DF = F.h;
    bool stored = use_au;
    bool after_full = false;  // the latest residual was a full FP64 evaluation
    for (;;) {
      // Incremental residual: after a sweep that started from a full FP64 residual r,
      // b - A(x + xc d) = b - (A x + xc A d) with A x kept in FP64 and A d the FP32
      // product of the correction, when its rounding estimate kIncrC u32 lam_max xc ||d||
      // is at most a quarter of the outer target (the estimate is added to ||r|| in the
      // convergence test).  At most one such update follows each full evaluation.
      bool incr = false;
      double rb = 0.0;
      if (!stored && after_full && h->opt.incr_resid && h->lam_max > 0 && D.slot[SL_AU]) {
        launch_dnorm2(P, h->st);
        launch_fin(h->sc64, nullptr, 0, nullptr, 0, D.part[PT_C], ew_block_count(P), FIN_DNORM, nullptr, h->st);
        CKH(h, cudaGetLastError());
        int rc = read_scalars(h);
        if (rc) return rc;
        const Scalars& s64 = h->host_sc[0];
        rb = kIncrC * std::ldexp(1.0, -24) * h->lam_max * h->host_sc[1].xcoef * std::sqrt(s64.dnorm2);
        incr = std::isfinite(rb) && rb <= 0.25 * std::sqrt(s64.tol2 * s64.ref2);
      }
      if (stored) {
        // initial residual already formed by the predictor from the stored A u; with an
        // increment warm start d, q = P A d (FP32) for the first inner solve's residual
        if (inner_guess) launch_apply<float>(F, PRE_PLAIN, SL_D, POST_APPLY, SL_Q, 1, 0, h->st);
        launch_fin(h->sc64, D.part[PT_B], ew_block_count(P), nullptr, 0, nullptr, 0, FIN_OUTER, h->sc32, h->st);
        after_full = false;
      } else if (incr) {
        launch_incr_begin(h->sc64, h->sc32, rb, h->st);
        launch_apply<float>(F, PRE_PLAIN, SL_D, POST_APPLY, SL_Q, 0, 0, h->st);
        launch_resid_incr(P, reinterpret_cast<const float*>(DF.slot[SL_Q]), 1, h->st);
        launch_fin(h->sc64, D.part[PT_A], ew_block_count(P), nullptr, 0, nullptr, 0, FIN_OUTER, h->sc32, h->st);
        ++incr_count;
        h->au_bound = rb;
        after_full = false;
      } else {
        // after an inner solve the residual pass first folds its FP32 correction into x
        launch_apply<double>(P, sweeps > 0 ? PRE_XUPD : PRE_PLAIN, SL_X, POST_RESID, 0, 1, 1, h->st);
        launch_fin(h->sc64, D.part[PT_A], P.g.blk_x, nullptr, 0, nullptr, 0, FIN_OUTER, h->sc32, h->st);
        ++outer;
        h->au_bound = 0.0;
        after_full = true;
      }
      h->last_resid_on_x = !stored;
      stored = false;
      CKH(h, cudaGetLastError());
      int rc = read_scalars(h);
      if (rc) return rc;
      if (h->host_sc[0].done) {
        status = h->host_sc[0].status;
        break;
      }
      if (sweeps >= h->opt.max_sweeps) {
        status = WFFT_ENOTCONV;
        break;
      }
      if (iters >= watchdog) {
        status = WFFT_ETIMEOUT;
        break;
      }
      ++sweeps;
      precond_start<float>(F, h->sc32, inner_guess && sweeps == 1 ? PRE_CONVD : PRE_CONV, 1, h->st);
      int it = 0;
      rc = pcg_loop<float>(h, F, h->sc32, 1, std::max(1, watchdog - iters), &it);
      iters += it;
      if (rc == WFFT_ETIMEOUT) {
        status = WFFT_ETIMEOUT;
        break;
      }
      if (rc) return rc;
      if (h->host_sc[1].status == WFFT_ENUMERIC) {
        status = WFFT_ENUMERIC;
        break;
      }
    }
  }
  const Scalars& s = h->host_sc[0];
  if (info) {
    info->iters = iters;
    info->outer_applies = outer;
    info->sweeps = sweeps;
    info->incr_resids = incr_count;
    info->ref = std::sqrt(s.ref2);
    info->rel_res = s.ref2 > 0 ? std::sqrt(s.rr / s.ref2) : 0.0;
  }
  return status;
}

static void fill_info_base(wfft_step_info* info) {
  if (!info) return;
  memset(info, 0, sizeof(*info));
}

__global__ static void k_add_delta(const Desc<double>* dd, const float* delta) {
  const Desc<double>& D = *dd;
  double* x = reinterpret_cast<double*>(D.slot[SL_X]);
  const long long tot = (long long)D.c * D.V;
  for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < tot;
       gi += (long long)gridDim.x * blockDim.x)
    x[gi] += (double)delta[gi];  // delta is 0 on the prescribed DOFs
}

extern "C" int wfft_step(wfft_handle* h, const double U[3], wfft_step_info* info) {
  ProfScope ps_(h);
  if (!h) return fail(nullptr, WFFT_EINVAL, "null handle");
  if (h->explicit_scheme) return fail(h, WFFT_EINVAL, "explicit-scheme handle: use wfft_explicit_step");
  if (!U) return fail(h, WFFT_EINVAL, "U is NULL");
  fill_info_base(info);
  const int warm = h->opt.warm_start;
  if (warm == WFFT_WARM_LEARNED && !h->net) return fail(h, WFFT_EINVAL, "no warm-start model loaded");
  Plan<double>& P = h->P64;
  const bool mixed = h->opt.precision == WFFT_MIXED;
  double Uv[3];
  map_U(h, U, Uv);
  // increment warm starts: x0 = u_{n-1} + delta (delta FP32, zero on Gamma); in a
  // mixed solve with the stored A u_{n-1} the increment is the initial guess of the
  // first FP32 inner solve, so the initial residual still needs no FP64 apply
  const bool delta_mode = warm == WFFT_WARM_LEARNED || (mixed && warm == WFFT_WARM_TAYLOR);
  const bool use_au = mixed && h->au_valid && (warm == WFFT_WARM_PREV || delta_mode);
  const double dU[3] = {Uv[0] - h->U_prev[0], Uv[1] - h->U_prev[1], Uv[2] - h->U_prev[2]};
  CKH(h, cudaEventRecord(h->ev0, h->st));
  // the stored A u may carry the rounding bound of an incremental update
  launch_begin(h->sc64, Uv, delta_mode ? WFFT_WARM_PREV : warm, h->opt.tol * h->opt.tol, h->opt.maxit, h->st,
               use_au ? 1 : 0, dU, h->opt.inner_floor > 0 ? h->opt.inner_floor : 0.0, use_au ? h->au_bound : 0.0);
  launch_begin(h->sc32, Uv, delta_mode ? WFFT_WARM_PREV : warm, h->opt.inner_tol * h->opt.inner_tol,
               h->opt.maxit, h->st);
  launch_predict(P, h->st);
  launch_fin(h->sc64, P.h.part[PT_A], ew_block_count(P), nullptr, 0, nullptr, 0, FIN_REF, nullptr, h->st);
  bool inner_guess = false;
  if (delta_mode) {
    WarmArgs wa;
    handle_warm_args(h, Uv, &wa, nullptr, nullptr);
    float* delta = mixed ? reinterpret_cast<float*>(h->P32.h.slot[SL_D]) : h->delta;
    net_warm(warm == WFFT_WARM_LEARNED ? h->net : nullptr, &h->nw, wa, delta, h->st);
    if (use_au) {
      inner_guess = true;
    } else {
      prof_launch(0, KK_NEWMARK, 20.0 * h->c * h->V, (double)h->c * h->V, h->st,
                  [&] { k_add_delta<<<ew_block_count(P), 256, 0, h->st>>>(P.d, delta); });
    }
  }
  h->last_resid_on_x = false;
  int status = solve_core(h, info, use_au, inner_guess);
  // a learned warm start whose tensor-core convolution gave up waiting: not committed
  if (warm == WFFT_WARM_LEARNED && status == WFFT_OK && net_conv_timed_out()) status = WFFT_ETIMEOUT;
  // the stored A x is A u_n only if the last residual evaluation ran on the final x
  h->au_valid = status == WFFT_OK && mixed && h->last_resid_on_x && !h->host_sc[0].zero_free;
  if (status == WFFT_OK) {
    for (int k = 0; k < 3; ++k) h->U_prev[k] = Uv[k];
    int rcw = wait_downloads(h, h->st);  // the corrector overwrites u, v, a
    if (rcw) return rcw;
    launch_correct(P, h->st);
    const int nb = ew_block_count(P);
    launch_fin(h->sc64, P.h.part[PT_A], nb, P.h.part[PT_B], nb, P.h.part[PT_C], nb, FIN_REACT, nullptr, h->st);
  launch_fin(h->sc64, P.h.part[PT_D], nb, P.h.part[PT_E], nb, nullptr, 0, FIN_ENERGY, nullptr, h->st);
    ++h->nstep;
  }
  CKH(h, cudaEventRecord(h->ev1, h->st));
  CKH(h, cudaGetLastError());
  int rc = read_scalars(h);
  if (rc) return rc;
  if (info) {
    info->status = status;
    if (status == WFFT_OK) put_reaction(h, h->host_sc[0].react, info->reaction);
    info->energy = status == WFFT_OK ? step_energy(h, h->host_sc[0], Uv, false) : 0.0;
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    info->ms = ms;
  }
  if (status != WFFT_OK) {
    char buf[128];
    snprintf(buf, sizeof buf, "step not committed (status %d)", status);
    return fail(h, status, buf);
  }
  return WFFT_OK;
}

namespace wfft {
// Device fields of a handle for the warm-start kernels (k_net.cu).
int handle_warm_args(wfft_handle* h, const double U[3], WarmArgs* a, cudaStream_t* st, int* device) {
  if (!h || !a) return WFFT_EINVAL;
  const Desc<double>& D = h->P64.h;
  const Desc<float>& F = h->P32.h;
  WarmArgs w{};
  w.n1 = h->n[0];
  w.n2 = h->n[1];
  w.n3 = h->n[2];
  w.c = h->c;
  w.V = h->V;
  w.u = reinterpret_cast<const double*>(D.slot[SL_U]);
  w.v = reinterpret_cast<const double*>(D.slot[SL_V]);
  w.a = reinterpret_cast<const double*>(D.slot[SL_A]);
  w.mask = h->has_mask ? D.mask : nullptr;
  w.phase = D.phase;
  w.ctab = F.ctab;
  w.cstride = h->ndim == 3 ? kCtabStride3 : kCtabStride2;
  w.rhotab = F.rhotab;
  // entries of the material row and of the 21-value mean stiffness for the features:
  // normal diagonal, shear diagonal (summed), normal off-diagonal (summed)
  const int nd3[3] = {0, 6, 11}, sh3[3] = {15, 18, 20}, of3[3] = {1, 2, 7};
  const int nd2[3] = {0, 3, -1}, sh2[3] = {5, -1, -1}, of2[3] = {1, -1, -1};
  const int nd2c[3] = {0, 6, -1}, sh2c[3] = {20, -1, -1}, of2c[3] = {1, -1, -1};
  const bool three = h->ndim == 3;
  double ssh = 0, sof = 0;
  for (int k = 0; k < 3; ++k) {
    w.nd_idx[k] = three ? nd3[k] : nd2[k];
    w.sh_idx[k] = three ? sh3[k] : sh2[k];
    w.of_idx[k] = three ? of3[k] : of2[k];
    const int ndc = three ? nd3[k] : nd2c[k], shc = three ? sh3[k] : sh2c[k], ofc = three ? of3[k] : of2c[k];
    w.inv_nd[k] = ndc >= 0 && h->cbar[ndc] > 0 ? (float)(1.0 / h->cbar[ndc]) : 0.f;
    if (shc >= 0) ssh += h->cbar[shc];
    if (ofc >= 0) sof += h->cbar[ofc];
  }
  w.inv_sh = ssh > 0 ? (float)(1.0 / ssh) : 0.f;
  w.inv_of = std::fabs(sof) > 1e-12 * std::fabs(h->cbar[0]) ? (float)(1.0 / sof) : 0.f;
  w.inv_rhobar = (float)(1.0 / h->rhobar);
  w.dt = h->dt;
  w.theta = h->theta;
  for (int k = 0; k < 3; ++k) w.Ug[k] = k < h->c ? U[k] : 0.0;
  *a = w;
  if (st) *st = h->st;
  if (device) {
    cudaPointerAttributes pa;
    *device = cudaPointerGetAttributes(&pa, D.slot[SL_U]) == cudaSuccess ? pa.device : -1;
  }
  return WFFT_OK;
}
}  // namespace wfft

extern "C" int wfft_set_model(wfft_handle* h, const void* blob, size_t bytes) {
  if (!h) return fail(nullptr, WFFT_EINVAL, "null handle");
  if (!blob && bytes == 0) {
    CKH(h, cudaStreamSynchronize(h->st));
    net_free(h->net);
    h->net = nullptr;
    return WFFT_OK;
  }
  CKH(h, cudaStreamSynchronize(h->st));
  NetDev* n = nullptr;
  std::string err;
  int rc = net_upload(blob, bytes, false, &n, &err);
  if (rc) return fail(h, rc, err);
  rc = net_work_alloc(&h->nw, h->V, n->d.hidden);
  if (rc) {
    net_free(n);
    return fail(h, rc, "warm-start work buffers");
  }
  if (h->opt.precision == WFFT_FP64 && !h->delta) {
    cudaError_t e = dalloc(h, &h->delta, (size_t)h->c * h->V * sizeof(float));
    if (e != cudaSuccess) {
      net_free(n);
      return fail(h, WFFT_ENOMEM, "warm-start increment buffer");
    }
  }
  net_free(h->net);
  h->net = n;
  return WFFT_OK;
}

__global__ static void k_keep_gamma(const Desc<double>* dd, double* x) {
  const Desc<double>& D = *dd;
  const long long tot = (long long)D.c * D.V;
  for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < tot;
       gi += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(gi / D.V);
    const long long vox = gi - (long long)k * D.V;
    if (!((D.mask[vox] >> k) & 1)) x[gi] = 0.0;
  }
}

extern "C" int wfft_solve(wfft_handle* h, const double* b, double* x, double tol, int maxit, wfft_step_info* info) {
  ProfScope ps_(h);
  if (!h) return fail(nullptr, WFFT_EINVAL, "null handle");
  if (h->explicit_scheme) return fail(h, WFFT_EINVAL, "explicit-scheme handle: use wfft_explicit_step");
  if (!b || !x) return fail(h, WFFT_EINVAL, "b and x are required");
  fill_info_base(info);
  h->au_valid = false;  // the residual evaluations below overwrite the stored A u
  Plan<double>& P = h->P64;
  const double t = tol > 0 ? tol : h->opt.tol;
  const int mi = maxit > 0 ? maxit : h->opt.maxit;
  const int saved = h->opt.maxit;
  h->opt.maxit = mi;
  const double U0[3] = {0, 0, 0};
  CKH(h, cudaEventRecord(h->ev0, h->st));
  launch_begin(h->sc64, U0, 0, t * t, mi, h->st);
  launch_begin(h->sc32, U0, 0, h->opt.inner_tol * h->opt.inner_tol, mi, h->st);
  int rcc = field_copy(h, P.h.slot[SL_B], b, cudaMemcpyHostToDevice);
  if (rcc) return rcc;
  // ref^2 = ||P(b - A x_Gamma)||^2: residual of x with its free DOFs zeroed
  rcc = field_copy(h, P.h.slot[SL_X], x, cudaMemcpyHostToDevice);
  if (rcc) return rcc;
  prof_launch(0, KK_NEWMARK, 16.0 * h->c * h->V, 0.0, h->st,
              [&] { k_keep_gamma<<<ew_block_count(P), 256, 0, h->st>>>(P.d, (double*)P.h.slot[SL_X]); });
  launch_apply<double>(P, PRE_PLAIN, SL_X, POST_RESID, 0, 1, 1, h->st);
  launch_fin(h->sc64, P.h.part[PT_A], P.g.blk_x, nullptr, 0, nullptr, 0, FIN_REF, nullptr, h->st);
  rcc = field_copy(h, P.h.slot[SL_X], x, cudaMemcpyHostToDevice);
  if (rcc) return rcc;
  int status = solve_core(h, info);
  h->opt.maxit = saved;
  if (h->host_sc[0].zero_free)
    prof_launch(0, KK_NEWMARK, 16.0 * h->c * h->V, 0.0, h->st,
                [&] { k_keep_gamma<<<ew_block_count(P), 256, 0, h->st>>>(P.d, (double*)P.h.slot[SL_X]); });
  CKH(h, cudaEventRecord(h->ev1, h->st));
  rcc = field_copy(h, x, P.h.slot[SL_X], cudaMemcpyDeviceToHost);
  if (rcc) return rcc;
  CKH(h, cudaStreamSynchronize(h->st));
  CKH(h, cudaGetLastError());
  if (info) {
    info->status = status;
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    info->ms = ms;
  }
  if (status != WFFT_OK) return fail(h, status, "solve did not converge");
  return WFFT_OK;
}

extern "C" int wfft_apply(wfft_handle* h, int precision, const void* p_dev, void* q_dev, int masked) {
  ProfScope ps_(h);
  if (!h || !p_dev || !q_dev) return fail(h, WFFT_EINVAL, "null argument");
  if (h->relabeled) return fail(h, WFFT_EUNSUPPORTED, "field calls on a grid with N1 = 1 (relabeled axes)");
  if (precision == WFFT_FP64) {
    launch_set_done(h->sc64, 0, h->st);
    CKH(h, set_ext(h->P64, p_dev, q_dev, h->st));
    launch_apply<double>(h->P64, PRE_PLAIN, SL_EXT_IN, POST_APPLY, SL_EXT_OUT, masked ? 1 : 0, 0, h->st);
  } else if (precision == WFFT_MIXED) {
    launch_set_done(h->sc32, 0, h->st);
    CKH(h, set_ext(h->P32, p_dev, q_dev, h->st));
    launch_apply<float>(h->P32, PRE_PLAIN, SL_EXT_IN, POST_APPLY, SL_EXT_OUT, masked ? 1 : 0, 0, h->st);
  } else {
    return fail(h, WFFT_EINVAL, "unknown precision");
  }
  CKH(h, cudaGetLastError());
  return WFFT_OK;
}

extern "C" int wfft_precond(wfft_handle* h, int precision, const void* r_dev, void* z_dev, int masked) {
  ProfScope ps_(h);
  if (h && h->relabeled) return fail(h, WFFT_EUNSUPPORTED, "field calls on a grid with N1 = 1 (relabeled axes)");
  if (!h || !r_dev || !z_dev) return fail(h, WFFT_EINVAL, "null argument");
  if (precision == WFFT_FP64) {
    launch_set_done(h->sc64, 0, h->st);
    CKH(h, set_ext(h->P64, r_dev, z_dev, h->st));
    launch_precond<double>(h->P64, PRE_PLAIN, SL_EXT_IN, SL_EXT_OUT, masked ? 1 : 0, h->st);
  } else if (precision == WFFT_MIXED) {
    launch_set_done(h->sc32, 0, h->st);
    CKH(h, set_ext(h->P32, r_dev, z_dev, h->st));
    launch_precond<float>(h->P32, PRE_PLAIN, SL_EXT_IN, SL_EXT_OUT, masked ? 1 : 0, h->st);
  } else {
    return fail(h, WFFT_EINVAL, "unknown precision");
  }
  CKH(h, cudaGetLastError());
  return WFFT_OK;
}

template <typename T>
static int rfft3_impl(wfft_handle* h, Plan<T>& P, Scalars* sc, int dir, int ncomp, const void* in, void* out) {
  const size_t sbytes = (size_t)ncomp * P.h.Vh * sizeof(cplx<T>);
  if (!rfft3_fits<T>(P, ncomp))
    return fail(h, WFFT_EUNSUPPORTED, "this many components on this x axis do not fit the transform's tiles");
  launch_set_done(sc, 0, h->st);
  if (dir < 0) {
    CKH(h, set_ext(P, in, out, h->st));
    launch_rfft3<T>(P, -1, ncomp, SL_EXT_IN, h->st);
    CKH(h, cudaMemcpyAsync(out, P.h.spec, sbytes, cudaMemcpyDeviceToDevice, h->st));
  } else {
    CKH(h, set_ext(P, out, out, h->st));
    CKH(h, cudaMemcpyAsync(P.h.spec, in, sbytes, cudaMemcpyDeviceToDevice, h->st));
    launch_rfft3<T>(P, +1, ncomp, SL_EXT_OUT, h->st);
  }
  CKH(h, cudaGetLastError());
  return WFFT_OK;
}

extern "C" int wfft_rfft3(wfft_handle* h, int precision, int dir, int ncomp, const void* in_dev, void* out_dev) {
  ProfScope ps_(h);
  if (!h || !in_dev || !out_dev) return fail(h, WFFT_EINVAL, "null argument");
  if (h->relabeled) return fail(h, WFFT_EUNSUPPORTED, "field calls on a grid with N1 = 1 (relabeled axes)");
  if (ncomp < 1 || ncomp > h->s || (dir != -1 && dir != 1)) return fail(h, WFFT_EINVAL, "bad ncomp or dir");
  if (precision == WFFT_FP64) return rfft3_impl<double>(h, h->P64, h->sc64, dir, ncomp, in_dev, out_dev);
  if (precision == WFFT_MIXED) return rfft3_impl<float>(h, h->P32, h->sc32, dir, ncomp, in_dev, out_dev);
  return fail(h, WFFT_EINVAL, "unknown precision");
}

// ---------------------------------------------------------------------------
// grouped steps of several handles: every pass is one launch over all
// instances that have not converged yet
// ---------------------------------------------------------------------------
namespace {

enum FinSlot {
  FJ_REF = 0, FJ_RES0, FJ_RZ0, FJ_ALPHA, FJ_BETA, FJ_OUTER_STORED, FJ_OUTER_RESID, FJ_REACT,
  FJ_RZ0_32, FJ_ALPHA_32, FJ_BETA_32, FJ_DNORM, FJ_OUTER_INCR, FJ_ENERGY, FJ_N
};

struct BatchCtx {
  std::vector<wfft_handle*> hs;
  int precision = -1;
  BatchLaunch<double> bl64;
  BatchLaunch<float> bl32;
  std::vector<void*> dev;  // device allocations of this context
  FinJob* fin[FJ_N] = {};
  BeginJob* begin64 = nullptr;
  BeginJob* begin32 = nullptr;
  Scalars* host = nullptr;  // pinned mirror: [i] = sc64 of instance i, [n + i] = sc32
  Scalars* const* dsrc = nullptr;  // device: sc64 pointers then sc32 pointers
  Scalars* dgather = nullptr;      // device: gathered copies
  const float* const* q32s = nullptr;  // device: FP32 operator output (SL_Q) of each instance
  double* rb_dev = nullptr;            // device / pinned host: rounding estimates of an
  double* rb_host = nullptr;           //   incremental residual, per instance
  std::vector<BeginJob> hb64, hb32;
  // CUDA graphs of one block of grouped PCG iterations per precision (captured lazily)
  cudaStream_t cap_st = nullptr;
  cudaGraphExec_t chunk[2] = {nullptr, nullptr};
  int chunk_iters[2] = {0, 0};
  long long chunk_launches[2] = {0, 0};
  ~BatchCtx() {
    for (int k = 0; k < 2; ++k)
      if (chunk[k]) cudaGraphExecDestroy(chunk[k]);
    if (cap_st) cudaStreamDestroy(cap_st);
    for (void* p : dev) cudaFree(p);
    if (host) cudaFreeHost(host);
    if (rb_host) cudaFreeHost(rb_host);
  }
};
BatchCtx* g_batch = nullptr;

template <typename T>
cudaError_t build_launch(BatchCtx& B, BatchLaunch<T>& bl, Plan<T> wfft_handle::*plan, std::vector<void*>& dev) {
  const int n = (int)B.hs.size();
  bl.n = n;
  bl.plans.clear();
  for (wfft_handle* h : B.hs) bl.plans.push_back(&(h->*plan));
  // every instance keeps its own column-tile widths (its tuned plan): a column class
  // is one group of instances per distinct width, each group its own grouped launch
  auto own_bx = [&](int i, int cls) {
    return std::max(1, bl.plans[i]->g.bx[(cls - GEO_COL0) / 5 + 1][(cls - GEO_COL0) % 5]);
  };
  std::vector<int> starts((size_t)NGEO * (n + 1));
  std::vector<std::vector<int>> gstarts;  // prefix sums of the column groups
  std::vector<std::pair<int, int>> gkey;  // (class, group index) of each gstarts entry
  for (int cls = 0; cls < NGEO; ++cls) {
    const bool col = cls >= GEO_COL0 && cls < GEO_EW;
    int acc = 0;
    size_t sm = 0;
    for (int i = 0; i < n; ++i) {
      const int bx = col ? own_bx(i, cls) : 1;
      starts[(size_t)cls * (n + 1) + i] = acc;
      acc += geo_blocks<T>(*bl.plans[i], cls, bx);
      sm = std::max(sm, geo_smem<T>(*bl.plans[i], cls, bx));
    }
    starts[(size_t)cls * (n + 1) + n] = acc;
    bl.total[cls] = acc;
    bl.sm[cls] = sm;
    if (!col) continue;
    std::vector<ColGroup<T>>& groups = bl.cols[cls - GEO_COL0];
    groups.clear();
    for (int i = 0; i < n; ++i) {
      const int bx = own_bx(i, cls);
      bool seen = false;
      for (const ColGroup<T>& g : groups) seen = seen || g.bx == bx;
      if (seen) continue;
      ColGroup<T> g;
      g.bx = bx;
      std::vector<int> st(n + 1);
      int a = 0;
      for (int j = 0; j < n; ++j) {
        st[j] = a;
        if (own_bx(j, cls) != bx) continue;
        a += geo_blocks<T>(*bl.plans[j], cls, bx);
        g.sm = std::max(g.sm, geo_smem<T>(*bl.plans[j], cls, bx));
        g.plans.push_back(bl.plans[j]);
      }
      st[n] = a;
      g.total = a;
      gkey.push_back({cls, (int)groups.size()});
      gstarts.push_back(st);
      groups.push_back(g);
    }
  }
  void *dstart = nullptr, *ddesc = nullptr;
  const size_t nstart = starts.size() + gstarts.size() * (size_t)(n + 1);
  cudaError_t e = cudaMalloc(&dstart, nstart * sizeof(int));
  if (e != cudaSuccess) return e;
  dev.push_back(dstart);
  for (const std::vector<int>& st : gstarts) starts.insert(starts.end(), st.begin(), st.end());
  e = cudaMemcpy(dstart, starts.data(), nstart * sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  for (int cls = 0; cls < NGEO; ++cls) bl.start[cls] = reinterpret_cast<int*>(dstart) + (size_t)cls * (n + 1);
  for (size_t k = 0; k < gkey.size(); ++k)
    bl.cols[gkey[k].first - GEO_COL0][gkey[k].second].start =
        reinterpret_cast<int*>(dstart) + (size_t)(NGEO + k) * (n + 1);
  std::vector<const Desc<T>*> descs;
  for (const Plan<T>* q : bl.plans) descs.push_back(q->d);
  e = cudaMalloc(&ddesc, descs.size() * sizeof(void*));
  if (e != cudaSuccess) return e;
  dev.push_back(ddesc);
  e = cudaMemcpy(ddesc, descs.data(), descs.size() * sizeof(void*), cudaMemcpyHostToDevice);
  bl.descs = reinterpret_cast<const Desc<T>* const*>(ddesc);
  return e;
}

template <typename T>
int blocks_of(const BatchLaunch<T>& bl, int i, int cls) {
  int bx = 1;
  if (cls >= GEO_COL0 && cls < GEO_EW) bx = std::max(1, bl.plans[i]->g.bx[(cls - GEO_COL0) / 5 + 1][(cls - GEO_COL0) % 5]);
  return geo_blocks<T>(*bl.plans[i], cls, bx);
}

int build_batch(std::vector<wfft_handle*>& hs, BatchCtx*& out, std::string& err) {
  BatchCtx* B = new BatchCtx();
  B->hs = hs;
  B->precision = hs[0]->opt.precision;
  const int n = (int)hs.size();
  cudaError_t e = build_launch<double>(*B, B->bl64, &wfft_handle::P64, B->dev);
  if (e == cudaSuccess) e = build_launch<float>(*B, B->bl32, &wfft_handle::P32, B->dev);
  std::vector<FinJob> jobs((size_t)FJ_N * n);
  for (int i = 0; i < n; ++i) {
    wfft_handle* h = hs[i];
    const Desc<double>& D = h->P64.h;
    const Desc<float>& F = h->P32.h;
    const int ew = blocks_of(B->bl64, i, GEO_EW), bx64 = blocks_of(B->bl64, i, GEO_X);
    const int pr64 = blocks_of(B->bl64, i, geo_col(D.opAxis, OP_PREC));
    const int bx32 = blocks_of(B->bl32, i, GEO_X), pr32 = blocks_of(B->bl32, i, geo_col(F.opAxis, OP_PREC));
    auto J = [&](int slot) -> FinJob& { return jobs[(size_t)slot * n + i]; };
    J(FJ_REF) = {h->sc64, D.part[PT_A], ew, nullptr, 0, nullptr, 0, nullptr};
    J(FJ_RES0) = {h->sc64, D.part[PT_A], bx64, nullptr, 0, nullptr, 0, nullptr};
    J(FJ_RZ0) = {h->sc64, nullptr, 0, D.part[PT_B], pr64, nullptr, 0, nullptr};
    J(FJ_ALPHA) = {h->sc64, D.part[PT_A], bx64, nullptr, 0, nullptr, 0, nullptr};
    J(FJ_BETA) = {h->sc64, D.part[PT_A], bx64, D.part[PT_B], pr64, nullptr, 0, nullptr};
    J(FJ_OUTER_STORED) = {h->sc64, D.part[PT_B], ew, nullptr, 0, nullptr, 0, h->sc32};
    J(FJ_OUTER_RESID) = {h->sc64, D.part[PT_A], bx64, nullptr, 0, nullptr, 0, h->sc32};
    J(FJ_REACT) = {h->sc64, D.part[PT_A], ew, D.part[PT_B], ew, D.part[PT_C], ew, nullptr};
    J(FJ_ENERGY) = {h->sc64, D.part[PT_D], ew, D.part[PT_E], ew, nullptr, 0, nullptr};
    J(FJ_RZ0_32) = {h->sc32, nullptr, 0, F.part[PT_B], pr32, nullptr, 0, nullptr};
    J(FJ_ALPHA_32) = {h->sc32, F.part[PT_A], bx32, nullptr, 0, nullptr, 0, nullptr};
    J(FJ_BETA_32) = {h->sc32, F.part[PT_A], bx32, F.part[PT_B], pr32, nullptr, 0, nullptr};
    J(FJ_DNORM) = {h->sc64, nullptr, 0, nullptr, 0, D.part[PT_C], ew, nullptr};
    J(FJ_OUTER_INCR) = {h->sc64, D.part[PT_A], ew, nullptr, 0, nullptr, 0, h->sc32};
  }
  if (e == cudaSuccess) {
    std::vector<Scalars*> ptrs(2 * n);
    for (int i = 0; i < n; ++i) {
      ptrs[i] = hs[i]->sc64;
      ptrs[n + i] = hs[i]->sc32;
    }
    void *dp = nullptr, *dg = nullptr;
    e = cudaMalloc(&dp, ptrs.size() * sizeof(Scalars*));
    if (e == cudaSuccess) {
      B->dev.push_back(dp);
      e = cudaMemcpy(dp, ptrs.data(), ptrs.size() * sizeof(Scalars*), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc(&dg, 2 * n * sizeof(Scalars));
    if (e == cudaSuccess) {
      B->dev.push_back(dg);
      B->dsrc = reinterpret_cast<Scalars* const*>(dp);
      B->dgather = reinterpret_cast<Scalars*>(dg);
    }
  }
  void* dj = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&dj, jobs.size() * sizeof(FinJob) + 2 * n * sizeof(BeginJob));
  if (e == cudaSuccess) {
    B->dev.push_back(dj);
    e = cudaMemcpy(dj, jobs.data(), jobs.size() * sizeof(FinJob), cudaMemcpyHostToDevice);
    for (int k = 0; k < FJ_N; ++k) B->fin[k] = reinterpret_cast<FinJob*>(dj) + (size_t)k * n;
    B->begin64 = reinterpret_cast<BeginJob*>(reinterpret_cast<FinJob*>(dj) + jobs.size());
    B->begin32 = B->begin64 + n;
  }
  if (e == cudaSuccess) e = cudaMallocHost(&B->host, 2 * n * sizeof(Scalars));
  if (e == cudaSuccess) e = cudaMallocHost(&B->rb_host, n * sizeof(double));
  if (e == cudaSuccess) {
    std::vector<const float*> q(n);
    for (int i = 0; i < n; ++i) q[i] = reinterpret_cast<const float*>(hs[i]->P32.h.slot[SL_Q]);
    void* dq = nullptr;
    e = cudaMalloc(&dq, n * sizeof(const float*) + n * sizeof(double));
    if (e == cudaSuccess) {
      B->dev.push_back(dq);
      e = cudaMemcpy(dq, q.data(), n * sizeof(const float*), cudaMemcpyHostToDevice);
      B->q32s = reinterpret_cast<const float* const*>(dq);
      B->rb_dev = reinterpret_cast<double*>(reinterpret_cast<char*>(dq) + n * sizeof(const float*));
    }
  }
  if (e != cudaSuccess) {
    err = std::string("batch context: ") + cudaGetErrorString(e);
    delete B;
    return WFFT_ECUDA;
  }
  B->hb64.resize(n);
  B->hb32.resize(n);
  out = B;
  return WFFT_OK;
}

int batch_read(BatchCtx& B, cudaStream_t st) {
  const int n = (int)B.hs.size();
  launch_gather_scalars(B.dsrc, B.dgather, 2 * n, st);
  cudaError_t e = cudaMemcpyAsync(B.host, B.dgather, 2 * n * sizeof(Scalars), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? WFFT_OK : WFFT_ECUDA;
}

bool all_done(const BatchCtx& B, int which) {
  const int n = (int)B.hs.size();
  for (int i = 0; i < n; ++i)
    if (!B.host[which * n + i].done) return false;
  return true;
}

// Lockstep PCG iterations of plan type T over all instances until every one is done.
template <typename T>
int batch_pcg(BatchCtx& B, const BatchLaunch<T>& bl, const Plan<T>& P0, int which, int fa, int fb, int budget,
              int check_every, cudaStream_t st) {
  const int n = (int)B.hs.size();
  wfft_handle* h0 = B.hs[0];
  auto block = [&](cudaStream_t s) {
    for (int i = 0; i < check_every; ++i) {
      launch_apply<T>(P0, PRE_PUPD, SL_P, POST_APPLY, SL_Q, 1, 1, s, &bl);
      launch_fin_batch(B.fin[fa], n, FIN_ALPHA, s);
      launch_precond<T>(P0, PRE_RUPD, SL_R, SL_Z, 1, s, &bl);
      launch_fin_batch(B.fin[fb], n, FIN_BETA, s);
    }
  };
  // as for single solves: the block is captured once per context and precision on an
  // internal stream and replayed (every argument points at device-resident descriptors,
  // job tables and scalars); not while profiling
  const bool graphs = h0->opt.use_graphs && !h0->prof.on;
  int launched = 0;
  for (;;) {
    if (graphs) {
      if (!B.chunk[which] || B.chunk_iters[which] != check_every) {
        if (B.chunk[which]) cudaGraphExecDestroy(B.chunk[which]);
        B.chunk[which] = nullptr;
        if (!B.cap_st && cudaStreamCreateWithFlags(&B.cap_st, cudaStreamNonBlocking) != cudaSuccess)
          return WFFT_ECUDA;
        const long long before = h0->prof.lifetime;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(B.cap_st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return WFFT_ECUDA;
        block(B.cap_st);
        const cudaError_t ec = cudaStreamEndCapture(B.cap_st, &g);
        if (ec != cudaSuccess || !g) {
          if (g) cudaGraphDestroy(g);
          return WFFT_ECUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&B.chunk[which], g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
          B.chunk[which] = nullptr;
          return WFFT_ECUDA;
        }
        B.chunk_iters[which] = check_every;
        B.chunk_launches[which] = h0->prof.lifetime - before;
        h0->prof.lifetime = before;
      }
      if (cudaGraphLaunch(B.chunk[which], st) != cudaSuccess) return WFFT_ECUDA;
      h0->prof.lifetime += B.chunk_launches[which];
    } else {
      block(st);
    }
    launched += check_every;
    if (cudaGetLastError() != cudaSuccess) return WFFT_ECUDA;
    if (batch_read(B, st)) return WFFT_ECUDA;
    if (all_done(B, which)) return WFFT_OK;
    if (launched >= budget) return WFFT_ETIMEOUT;
  }
}

}  // namespace

extern "C" int wfft_batch_step(wfft_handle** hs, int n, const double* U, wfft_step_info* infos) {
  if (!hs || n < 0 || (n > 0 && !U)) return fail(nullptr, WFFT_EINVAL, "bad batch arguments");
  if (n == 0) return WFFT_OK;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return fail(nullptr, WFFT_EINVAL, "null handle in batch");
    if (hs[i]->explicit_scheme) return fail(nullptr, WFFT_EINVAL, "explicit-scheme handles step with wfft_explicit_step");
  }
  wfft_handle* h0 = hs[0];
  // the grouped path needs one structure: same precision, dimensionality, pass
  // sequence, stream and warm start; otherwise the handles step one by one
  bool grouped = n > 1;
  for (int i = 1; i < n && grouped; ++i) {
    wfft_handle* h = hs[i];
    grouped = h->opt.precision == h0->opt.precision && h->ndim == h0->ndim && h->st == h0->st &&
              h->P64.h.midAxis == h0->P64.h.midAxis && h->P64.h.opAxis == h0->P64.h.opAxis &&
              h->opt.warm_start == h0->opt.warm_start && h->opt.warm_start != WFFT_WARM_LEARNED;
  }
  if (!grouped) {
    int first = WFFT_OK;
    for (int i = 0; i < n; ++i) {
      int rc = wfft_step(hs[i], U + 3 * i, infos ? &infos[i] : nullptr);
      if (rc && !first) first = rc;
    }
    return first;
  }
  std::vector<wfft_handle*> v(hs, hs + n);
  if (!g_batch || g_batch->hs != v || g_batch->precision != h0->opt.precision) {
    delete g_batch;
    g_batch = nullptr;
    std::string err;
    int rc = build_batch(v, g_batch, err);
    if (rc) return fail(nullptr, rc, err);
  }
  BatchCtx& B = *g_batch;
  cudaStream_t st = h0->st;
  ProfScope ps_(h0);
  const bool mixed = h0->opt.precision == WFFT_MIXED;
  bool use_au = mixed && h0->opt.warm_start == WFFT_WARM_PREV;
  for (int i = 0; i < n; ++i) use_au = use_au && hs[i]->au_valid;
  for (int i = 0; i < n; ++i) {
    wfft_handle* h = hs[i];
    double Uv[3];
    map_U(h, U + 3 * i, Uv);
    BeginJob& b = B.hb64[i];
    b.sc = h->sc64;
    for (int k = 0; k < 3; ++k) {
      b.U[k] = Uv[k];
      b.dU[k] = Uv[k] - h->U_prev[k];
    }
    b.warm = h->opt.warm_start;
    b.tol2 = h->opt.tol * h->opt.tol;
    b.maxit = h->opt.maxit;
    b.use_au = use_au ? 1 : 0;
    b.rb = use_au ? h->au_bound : 0.0;
    B.hb32[i] = b;
    B.hb32[i].sc = h->sc32;
    B.hb32[i].tol2 = h->opt.inner_tol * h->opt.inner_tol;
    B.hb32[i].use_au = 0;
    B.hb32[i].rb = 0.0;
  }
  CKH(h0, cudaEventRecord(h0->ev0, st));
  CKH(h0, cudaMemcpyAsync(B.begin64, B.hb64.data(), n * sizeof(BeginJob), cudaMemcpyHostToDevice, st));
  CKH(h0, cudaMemcpyAsync(B.begin32, B.hb32.data(), n * sizeof(BeginJob), cudaMemcpyHostToDevice, st));
  launch_begin_batch(B.begin64, n, st);
  launch_begin_batch(B.begin32, n, st);
  const Plan<double>& P0 = h0->P64;
  const Plan<float>& F0 = h0->P32;
  launch_predict(P0, st, &B.bl64);
  launch_fin_batch(B.fin[FJ_REF], n, FIN_REF, st);
  const int watchdog = h0->opt.watchdog_iters > 0 ? h0->opt.watchdog_iters : 4 * h0->opt.maxit;
  std::vector<int> iters(n, 0), outer(n, 0), sweeps(n, 0), incrs(n, 0);
  std::vector<double> last_rb(n, 0.0);
  int status_all = WFFT_OK;
  bool last_resid_on_x = false;
  if (!mixed) {
    launch_apply<double>(P0, PRE_PLAIN, SL_X, POST_RESID, 0, 1, 1, st, &B.bl64);
    launch_fin_batch(B.fin[FJ_RES0], n, FIN_RES0, st);
    launch_precond<double>(P0, PRE_PLAIN, SL_R, SL_Z, 1, st, &B.bl64);
    launch_fin_batch(B.fin[FJ_RZ0], n, FIN_RZ0, st);
    int rc = batch_pcg<double>(B, B.bl64, P0, 0, FJ_ALPHA, FJ_BETA, watchdog, h0->opt.check_every, st);
    if (rc == WFFT_ETIMEOUT) status_all = WFFT_ETIMEOUT;
    else if (rc) return fail(h0, rc, "batch solve failed");
    for (int i = 0; i < n; ++i) {
      iters[i] = B.host[i].iter;
      outer[i] = 1;
    }
  } else {
    bool stored = use_au;
    bool after_full = false;  // the latest residual was a full FP64 evaluation
    int sweep = 0, total_inner = 0;
    std::vector<char> active(n, 1);
    for (;;) {
      // incremental residual (as for single solves), taken only when every unfinished
      // instance's rounding estimate is within a quarter of its target
      bool incr = false;
      if (!stored && after_full && h0->opt.incr_resid) {
        launch_dnorm2(P0, st, &B.bl64);
        launch_fin_batch(B.fin[FJ_DNORM], n, FIN_DNORM, st);
        if (cudaGetLastError() != cudaSuccess || batch_read(B, st)) return fail(h0, WFFT_ECUDA, "batch solve failed");
        incr = true;
        for (int i = 0; i < n; ++i) {
          const Scalars& s64 = B.host[i];
          B.rb_host[i] = 0.0;
          if (s64.done) continue;
          const double rb =
              kIncrC * std::ldexp(1.0, -24) * hs[i]->lam_max * B.host[n + i].xcoef * std::sqrt(s64.dnorm2);
          B.rb_host[i] = rb;
          if (!(hs[i]->lam_max > 0) || !std::isfinite(rb) || !(rb <= 0.25 * std::sqrt(s64.tol2 * s64.ref2)))
            incr = false;
        }
      }
      if (stored) {
        launch_fin_batch(B.fin[FJ_OUTER_STORED], n, FIN_OUTER, st);
        after_full = false;
      } else if (incr) {
        CKH(h0, cudaMemcpyAsync(B.rb_dev, B.rb_host, n * sizeof(double), cudaMemcpyHostToDevice, st));
        launch_incr_begin_batch(B.dsrc, n, B.rb_dev, st);
        launch_apply<float>(F0, PRE_PLAIN, SL_D, POST_APPLY, SL_Q, 0, 0, st, &B.bl32);
        launch_resid_incr(P0, nullptr, 1, st, &B.bl64, B.q32s);
        launch_fin_batch(B.fin[FJ_OUTER_INCR], n, FIN_OUTER, st);
        for (int i = 0; i < n; ++i)
          if (active[i]) {
            ++incrs[i];
            last_rb[i] = B.rb_host[i];
          }
        after_full = false;
      } else {
        launch_apply<double>(P0, sweep > 0 ? PRE_XUPD : PRE_PLAIN, SL_X, POST_RESID, 0, 1, 1, st, &B.bl64);
        launch_fin_batch(B.fin[FJ_OUTER_RESID], n, FIN_OUTER, st);
        for (int i = 0; i < n; ++i) {
          outer[i] += active[i];
          if (active[i]) last_rb[i] = 0.0;
        }
        after_full = true;
      }
      last_resid_on_x = !stored;
      stored = false;
      if (cudaGetLastError() != cudaSuccess || batch_read(B, st)) return fail(h0, WFFT_ECUDA, "batch solve failed");
      for (int i = 0; i < n; ++i) active[i] = !B.host[i].done;
      if (all_done(B, 0)) break;
      if (sweep >= h0->opt.max_sweeps) {
        status_all = WFFT_ENOTCONV;
        break;
      }
      if (total_inner >= watchdog) {
        status_all = WFFT_ETIMEOUT;
        break;
      }
      ++sweep;
      for (int i = 0; i < n; ++i) sweeps[i] += active[i];
      launch_precond<float>(F0, PRE_CONV, SL_R, SL_Z, 1, st, &B.bl32);
      launch_fin_batch(B.fin[FJ_RZ0_32], n, FIN_RZ0, st);
      int rc = batch_pcg<float>(B, B.bl32, F0, 1, FJ_ALPHA_32, FJ_BETA_32, std::max(1, watchdog - total_inner),
                                h0->opt.check_every, st);
      int mx = 0;
      for (int i = 0; i < n; ++i)
        if (active[i]) {
          iters[i] += B.host[n + i].iter;
          mx = std::max(mx, B.host[n + i].iter);
        }
      total_inner += mx;
      if (rc == WFFT_ETIMEOUT) {
        status_all = WFFT_ETIMEOUT;
        break;
      }
      if (rc) return fail(h0, rc, "batch solve failed");
    }
  }
  // instances that did not finish fail (not committed); the corrector skips them
  std::vector<char> closed(n, 0);
  for (int i = 0; i < n; ++i) closed[i] = !B.host[i].done;
  launch_fin_batch(B.fin[FJ_REF], n, FIN_CLOSE, st);
  for (int i = 0; i < n; ++i) {
    int rcw = wait_downloads(hs[i], st);
    if (rcw) return rcw;
  }
  launch_correct(P0, st, &B.bl64);
  launch_fin_batch(B.fin[FJ_REACT], n, FIN_REACT, st);
  launch_fin_batch(B.fin[FJ_ENERGY], n, FIN_ENERGY, st);
  CKH(h0, cudaEventRecord(h0->ev1, st));
  if (batch_read(B, st)) return fail(h0, WFFT_ECUDA, "batch solve failed");
  float ms = 0;
  cudaEventElapsedTime(&ms, h0->ev0, h0->ev1);
  int first = WFFT_OK;
  for (int i = 0; i < n; ++i) {
    wfft_handle* h = hs[i];
    const Scalars& s64 = B.host[i];
    int st_i = s64.status;
    if (closed[i] && status_all != WFFT_OK) st_i = status_all;
    if (st_i == WFFT_OK) {
      ++h->nstep;
      for (int k = 0; k < 3; ++k) h->U_prev[k] = B.hb64[i].U[k];
    }
    h->au_valid = st_i == WFFT_OK && mixed && last_resid_on_x && !s64.zero_free;
    h->au_bound = last_rb[i];
    if (infos) {
      wfft_step_info& in = infos[i];
      memset(&in, 0, sizeof(in));
      in.status = st_i;
      in.iters = iters[i];
      in.outer_applies = outer[i];
      in.sweeps = sweeps[i];
      in.incr_resids = incrs[i];
      in.ref = std::sqrt(s64.ref2);
      in.rel_res = s64.ref2 > 0 ? std::sqrt(s64.rr / s64.ref2) : 0.0;
      if (st_i == WFFT_OK) put_reaction(h, s64.react, in.reaction);
      in.energy = st_i == WFFT_OK ? step_energy(h, s64, B.hb64[i].U, false) : 0.0;
      in.ms = ms;
    }
    if (st_i != WFFT_OK && !first) first = st_i;
  }
  return first;
}

extern "C" int wfft_profile(wfft_handle* h, int enable) {
  if (!h) return fail(nullptr, WFFT_EINVAL, "null handle");
  CKH(h, cudaStreamSynchronize(h->st));
  h->prof.collect();
  if (enable) {
    h->prof.reset();
    h->prof.on = true;
  } else {
    h->prof.on = false;
  }
  return WFFT_OK;
}

extern "C" int wfft_profile_read(wfft_handle* h, int precision, int kind, long long* launches, long long* timed,
                                 double* ms, double* alg_bytes, double* alg_flops) {
  if (!h || (precision != WFFT_FP64 && precision != WFFT_MIXED) || kind < 0 || kind >= KK_NKIND)
    return fail(h, WFFT_EINVAL, "bad profile query");
  CKH(h, cudaStreamSynchronize(h->st));
  h->prof.collect();
  const int p = precision == WFFT_FP64 ? 0 : 1;
  if (launches) *launches = h->prof.launches[p][kind];
  if (timed) *timed = h->prof.timed[p][kind];
  if (ms) *ms = h->prof.ms[p][kind];
  if (alg_bytes) *alg_bytes = h->prof.bytes[p][kind];
  if (alg_flops) *alg_flops = h->prof.flops[p][kind];
  return WFFT_OK;
}

extern "C" int wfft_launch_count(const wfft_handle* h, long long* launches) {
  if (!h || !launches) return fail(nullptr, WFFT_EINVAL, "null argument");
  *launches = h->prof.lifetime;
  return WFFT_OK;
}

// ---------------------------------------------------------------------------
// autotuner: radix decomposition of each axis and column-tile width of each column
// pass, timed on the handle's own grid and device
// ---------------------------------------------------------------------------
namespace {
struct TunedPlan {
  AxisPlan ax[3];
  int bx[3][5];
  int xelems;
};
std::mutex g_tune_mu;
std::map<std::array<int, 6>, TunedPlan> g_tuned;  // (precision, ndim, N1, N2, N3, device)

// one operator application + one preconditioner application on the Krylov scratch vectors
template <typename T>
float time_iteration(wfft_handle* h, Plan<T>& P, int reps) {
  launch_set_done(P.h.sc, 0, h->st);
  launch_apply<T>(P, PRE_PLAIN, SL_P, POST_APPLY, SL_Q, 1, 0, h->st);
  cudaEventRecord(h->ev0, h->st);
  for (int r = 0; r < reps; ++r) {
    launch_apply<T>(P, PRE_NONE, SL_P, POST_APPLY, SL_Q, 1, 0, h->st);
    launch_precond_part_impl<T>(P, 0, PRE_PLAIN, SL_Q, 1, h->st);
    launch_precond_part_impl<T>(P, 1, 0, 0, 1, h->st);
  }
  cudaEventRecord(h->ev1, h->st);
  float ms = 1e30f;
  if (cudaEventSynchronize(h->ev1) != cudaSuccess || cudaEventElapsedTime(&ms, h->ev0, h->ev1) != cudaSuccess)
    ms = 1e30f;
  return ms;
}

template <typename T>
bool ops_of_axis(const Desc<T>& D, int axis, int op) {
  if (axis == D.opAxis) return op == OP_GRAD || op == OP_DIV || op == OP_PREC;
  if (axis == D.midAxis) return op == OP_FWD || op == OP_INV;
  return false;
}

template <typename T>
int tune_plan(wfft_handle* h, Plan<T>& P, int prec, int reps, int* changed) {
  Desc<T>& D = P.h;
  int dev = 0;
  cudaGetDevice(&dev);
  const std::array<int, 6> key{prec, h->ndim, h->n[0], h->n[1], h->n[2], dev};
  TunedPlan before;
  for (int a = 0; a < 3; ++a) {
    before.ax[a] = D.ax[a];
    for (int op = 0; op < 5; ++op) before.bx[a][op] = P.g.bx[a][op];
  }
  before.xelems = P.g.xelems;
  TunedPlan best;
  bool cached = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      best = it->second;
      cached = true;
    }
  }
  if (!cached) {
    // 1. radix decomposition, axis by axis
    for (int a = 0; a < 3; ++a) {
      const std::vector<AxisPlan> cands = factor_candidates(h->n[a], true);
      if (h->n[a] == 1 || cands.size() < 2) continue;
      AxisPlan keep = D.ax[a];
      float tbest = 1e30f;
      for (const AxisPlan& c : cands) {
        D.ax[a] = c;
        plan_geometry<T>(P);
        if (!P.g.fits || P.g.max_blocks > h->nparts) continue;  // partial-sum arrays are sized at creation
        CKH(h, upload_desc(P));
        const float t = time_iteration<T>(h, P, reps);
        if (t < tbest) {
          tbest = t;
          keep = c;
        }
      }
      D.ax[a] = keep;
      plan_geometry<T>(P);
      CKH(h, upload_desc(P));
    }
    // 2. x-pass tile size (complex elements per block; larger tiles keep more loads in
    //    flight and more threads busy in the FFT stages, at the cost of shared memory)
    {
      const int keep0 = P.g.xelems;
      int keep = keep0;
      float tbest = 1e30f;
      for (int xe : {1024, 2048, 4096, kXReg | 2048, kXReg | 4096}) {
        P.g.xelems = xe;
        plan_geometry<T>(P);
        if (!P.g.fits || P.g.max_blocks > h->nparts) continue;
        CKH(h, upload_desc(P));
        const float t = time_iteration<T>(h, P, reps);
        if (t < tbest) {
          tbest = t;
          keep = xe;
        }
      }
      P.g.xelems = tbest < 1e30f ? keep : keep0;
      plan_geometry<T>(P);
      CKH(h, upload_desc(P));
    }
    // 3. column-tile widths, pass by pass
    for (int a = 1; a <= 2; ++a)
      for (int op = 0; op < 5; ++op) {
        if (!ops_of_axis(D, a, op)) continue;
        int keep = P.g.bx[a][op];
        float tbest = 1e30f;
        for (int bx : {1, 2, 4, 8, 16, kColReg | 4, kColReg | 8, kColReg | 16}) {
          if (!col_bx_feasible<T>(P, a, op, bx)) continue;
          set_col_bx<T>(P, a, op, bx);
          const float t = time_iteration<T>(h, P, reps);
          if (t < tbest) {
            tbest = t;
            keep = bx;
          }
        }
        set_col_bx<T>(P, a, op, keep);
      }
    for (int a = 0; a < 3; ++a) {
      best.ax[a] = D.ax[a];
      for (int op = 0; op < 5; ++op) best.bx[a][op] = P.g.bx[a][op];
    }
    best.xelems = P.g.xelems;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best;
  } else {
    for (int a = 0; a < 3; ++a) D.ax[a] = best.ax[a];
    P.g.xelems = best.xelems;
    plan_geometry<T>(P);
    if (!P.g.fits || P.g.max_blocks > h->nparts) {
      for (int a = 0; a < 3; ++a) D.ax[a] = before.ax[a];
      P.g.xelems = before.xelems;
      plan_geometry<T>(P);
    } else {
      for (int a = 1; a <= 2; ++a)
        for (int op = 0; op < 5; ++op)
          if (ops_of_axis(D, a, op) && col_bx_feasible<T>(P, a, op, best.bx[a][op]))
            set_col_bx<T>(P, a, op, best.bx[a][op]);
    }
    CKH(h, upload_desc(P));
  }
  for (int a = 0; a < 3; ++a) {
    bool same = D.ax[a].n == before.ax[a].n;
    for (int r = 0; r < 7; ++r) same = same && D.ax[a].cnt[r] == before.ax[a].cnt[r];
    if (!same) ++*changed;
    for (int op = 0; op < 5; ++op)
      if (ops_of_axis(D, a, op) && P.g.bx[a][op] != before.bx[a][op]) ++*changed;
  }
  if (P.g.xelems != before.xelems) ++*changed;
  CKH(h, cudaStreamSynchronize(h->st));
  return WFFT_OK;
}
}  // namespace

extern "C" int wfft_autotune(wfft_handle* h, int reps, int* changed) {
  if (!h) return fail(nullptr, WFFT_EINVAL, "null handle");
  if (h->prof.on) return fail(h, WFFT_EINVAL, "switch profiling off before tuning");
  ProfScope ps_(h);
  int ch = 0;
  const int r = reps > 0 ? reps : 3;
  CKH(h, cudaStreamSynchronize(h->st));
  int rc = tune_plan<double>(h, h->P64, 0, r, &ch);
  if (rc == WFFT_OK && h->opt.precision == WFFT_MIXED) rc = tune_plan<float>(h, h->P32, 1, r, &ch);
  // graphs captured with the old plan are stale
  for (int k = 0; k < 2; ++k)
    if (h->chunk[k]) {
      cudaGraphExecDestroy(h->chunk[k]);
      h->chunk[k] = nullptr;
    }
  if (changed) *changed = ch;
  return rc;
}

// ---------------------------------------------------------------------------
// explicit central-difference scheme (Sec. 2.3)
// ---------------------------------------------------------------------------
extern "C" int wfft_explicit_step(wfft_handle* h, const double Udot[3], wfft_step_info* info) {
  ProfScope ps_(h);
  if (!h) return fail(nullptr, WFFT_EINVAL, "null handle");
  if (!h->explicit_scheme) return fail(h, WFFT_EINVAL, "not an explicit-scheme handle (create it with beta = 0, gamma = 1/2)");
  if (!Udot) return fail(h, WFFT_EINVAL, "Udot is NULL");
  fill_info_base(info);
  Plan<double>& P = h->P64;
  double Uv[3];
  map_U(h, Udot, Uv);
  CKH(h, cudaEventRecord(h->ev0, h->st));
  launch_set_done(h->sc64, 0, h->st);
  {
    int rcw = wait_downloads(h, h->st);  // the explicit predictor overwrites u
    if (rcw) return rcw;
  }
  launch_explicit_predict(P, h->st);
  // q = -div(C : grad^s u_n), every DOF (unmasked)
  launch_apply<double>(P, PRE_PLAIN, SL_U, POST_PREC, SL_Q, 0, 0, h->st);
  launch_explicit_update(P, Uv, h->st);
  const int nb = ew_block_count(P);
  launch_fin(h->sc64, P.h.part[PT_A], nb, P.h.part[PT_B], nb, P.h.part[PT_C], nb, FIN_REACT, nullptr, h->st);
  launch_fin(h->sc64, P.h.part[PT_D], nb, P.h.part[PT_E], nb, nullptr, 0, FIN_ENERGY, nullptr, h->st);
  CKH(h, cudaEventRecord(h->ev1, h->st));
  CKH(h, cudaGetLastError());
  int rc = read_scalars(h);
  if (rc) return rc;
  h->au_valid = false;
  ++h->nstep;
  if (info) {
    info->status = WFFT_OK;
    info->outer_applies = 1;
    put_reaction(h, h->host_sc[0].react, info->reaction);
    info->energy = step_energy(h, h->host_sc[0], Uv, true);
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    info->ms = ms;
  }
  return WFFT_OK;
}

extern "C" int wfft_explicit_dt(int ndim, const double h[3], const double* C, const double* rho, long long nrows,
                                double* dt_max) {
  if ((ndim != 2 && ndim != 3) || !h || !C || !rho || nrows < 1 || !dt_max)
    return fail(nullptr, WFFT_EINVAL, "ndim 2 or 3, h, C, rho, nrows >= 1 and dt_max are required");
  double xi[3] = {0, 0, 0};
  for (int i = 0; i < ndim; ++i) {
    if (!(h[i] > 0)) return fail(nullptr, WFFT_EINVAL, "voxel sizes must be > 0");
    xi[i] = 3.141592653589793238462643383279502884 / h[i];  // N_i pi / L_i with L_i = N_i h_i
  }
  double w2 = 0.0;
  for (long long r = 0; r < nrows; ++r) {
    if (!(rho[r] > 0)) return fail(nullptr, WFFT_EINVAL, "rho must be > 0");
    w2 = std::max(w2, acoustic_max_eig(C + 21 * r, ndim, xi) / rho[r]);
  }
  if (!(w2 > 0)) return fail(nullptr, WFFT_EINVAL, "the stiffness gives no positive wave speed");
  *dt_max = 2.0 / std::sqrt(w2);
  return WFFT_OK;
}

extern "C" int wfft_operator_bound(int ndim, const int n[3], const double h[3], const double* C, const double* rho,
                                   long long nrows, double theta, double* lam_max) {
  if ((ndim != 2 && ndim != 3) || !n || !h || !C || !rho || nrows < 1 || !lam_max || !(theta >= 0))
    return fail(nullptr, WFFT_EINVAL, "ndim 2 or 3, n, h, C, rho, nrows >= 1, theta >= 0 and lam_max are required");
  for (int i = 0; i < ndim; ++i)
    if (n[i] < 1 || !(h[i] > 0)) return fail(nullptr, WFFT_EINVAL, "grid sizes and voxel sizes must be > 0");
  for (long long r = 0; r < nrows; ++r)
    if (!(rho[r] > 0)) return fail(nullptr, WFFT_EINVAL, "rho must be > 0");
  *lam_max = operator_max_eig_bound(ndim, n, h, C, rho, nrows, theta);
  return WFFT_OK;
}

extern "C" int wfft_axis_plan(int n, int cnt[7], int* prime) {
  if (!cnt || !prime) return fail(nullptr, WFFT_EINVAL, "cnt and prime are required");
  AxisPlan pl;
  if (!factorize(n, pl))
    return fail(nullptr, WFFT_EUNSUPPORTED,
                "axis lengths must be 1..2048 with prime factors 2, 3, 5, 7 and at most one other prime, up to 127");
  for (int r = 0; r < 7; ++r) cnt[r] = pl.cnt[r];
  *prime = pl.prime;
  return WFFT_OK;
}

namespace {
template <typename T>
int set_radix_plan(wfft_handle* h, Plan<T>& P, int axis, const AxisPlan& pl) {
  Desc<T>& D = P.h;
  const AxisPlan old = D.ax[axis];
  D.ax[axis] = pl;
  plan_geometry<T>(P);
  if (!P.g.fits || P.g.max_blocks > h->nparts) {
    const bool fits = P.g.fits;
    D.ax[axis] = old;
    plan_geometry<T>(P);
    return fail(h, WFFT_EINVAL, fits ? "this decomposition needs more partial-sum slots than the handle has"
                                     : "this decomposition's stages do not fit the passes' tiles");
  }
  CKH(h, cudaStreamSynchronize(h->st));
  CKH(h, upload_desc(P));
  for (int k = 0; k < 2; ++k)
    if (h->chunk[k]) {
      cudaGraphExecDestroy(h->chunk[k]);
      h->chunk[k] = nullptr;
    }
  return WFFT_OK;
}
}  // namespace

extern "C" int wfft_set_radix(wfft_handle* h, int precision, int axis, const int cnt[7]) {
  if (!h) return fail(nullptr, WFFT_EINVAL, "null handle");
  if ((precision != WFFT_FP64 && precision != WFFT_MIXED) || axis < 0 || axis > 2 || !cnt)
    return fail(h, WFFT_EINVAL, "precision WFFT_FP64 / WFFT_MIXED, axis 0..2 and cnt are required");
  if (h->prof.on) return fail(h, WFFT_EINVAL, "switch profiling off before changing plans");
  static const int rad[7] = {8, 4, 2, 3, 5, 7, 16};
  AxisPlan pl;
  pl.n = h->n[axis];
  pl.prime = axis_prime(h->n[axis]);  // the general prime stage is implied by the axis length
  long long prod = pl.prime > 0 ? pl.prime : 1;
  for (int r = 0; r < 7; ++r) {
    if (cnt[r] < 0 || cnt[r] > 16) return fail(h, WFFT_EINVAL, "stage counts must be 0..16");
    pl.cnt[r] = cnt[r];
    for (int k = 0; k < cnt[r]; ++k) prod *= rad[r];
  }
  if (prod != h->n[axis])
    return fail(h, WFFT_EINVAL,
                "the stages' radices (times the prime factor above 7, if any) must multiply to the axis length");
  ProfScope ps_(h);
  return precision == WFFT_FP64 ? set_radix_plan<double>(h, h->P64, axis, pl)
                                : set_radix_plan<float>(h, h->P32, axis, pl);
}

// ---------------------------------------------------------------------------
// Green's-matrix treatment of Gamma (Sec. 2.2.3, Eqs. f_discrete, G, Vt,
// L-determination_ND; Alg. 2)
// ---------------------------------------------------------------------------
namespace {
// x <- A^-1 b without the projection P (the unconstrained system of the Green's
// functions), PCG from the guess in SL_X to tol * ||b||; b in SL_B.
int green_solve(wfft_handle* h, int* iters) {
  Plan<double>& P = h->P64;
  const Desc<double>& D = P.h;
  h->solve_masked = 0;
  const double zero3[3] = {0.0, 0.0, 0.0};
  launch_begin(h->sc64, zero3, 0, h->opt.tol * h->opt.tol, h->opt.maxit, h->st);
  launch_green_norm2(P, reinterpret_cast<const double*>(D.slot[SL_B]), h->st);
  launch_fin(h->sc64, D.part[PT_A], ew_block_count(P), nullptr, 0, nullptr, 0, FIN_REF, nullptr, h->st);
  launch_apply<double>(P, PRE_PLAIN, SL_X, POST_RESID, 0, 0, 1, h->st);
  launch_fin(h->sc64, D.part[PT_A], P.g.blk_x, nullptr, 0, nullptr, 0, FIN_RES0, nullptr, h->st);
  precond_start<double>(P, h->sc64, PRE_PLAIN, 0, h->st);
  const int watchdog = h->opt.watchdog_iters > 0 ? h->opt.watchdog_iters : 4 * h->opt.maxit;
  int rc = pcg_loop<double>(h, P, h->sc64, 0, watchdog, iters);
  h->solve_masked = 1;
  if (rc == WFFT_OK && h->host_sc[0].status) rc = h->host_sc[0].status;
  return rc;
}
}  // namespace

extern "C" int wfft_green_setup(wfft_handle* h, long long max_dofs) {
  ProfScope ps_(h);
  if (!h) return fail(nullptr, WFFT_EINVAL, "null handle");
  if (h->explicit_scheme || h->opt.precision != WFFT_FP64)
    return fail(h, WFFT_EINVAL, "the Green's-matrix mode needs an FP64 implicit handle");
  if (!h->has_mask) return fail(h, WFFT_EINVAL, "no prescribed DOFs");
  if (h->green_n) return WFFT_OK;
  const long long cap = max_dofs > 0 ? max_dofs : 4096;
  Plan<double>& P = h->P64;
  const Desc<double>& D = P.h;
  const long long V = h->V;
  // prescribed DOF list k V + vox in ascending order, from the per-voxel mask bits
  std::vector<uint8_t> mb((size_t)V);
  CKH(h, cudaMemcpy(mb.data(), D.mask, (size_t)V, cudaMemcpyDeviceToHost));
  std::vector<long long> idx;
  for (int k = 0; k < h->c; ++k)
    for (long long v = 0; v < V; ++v)
      if ((mb[v] >> k) & 1) idx.push_back((long long)k * V + v);
  const long long n = (long long)idx.size();
  if (n > cap) {
    char buf[160];
    snprintf(buf, sizeof buf, "%lld prescribed DOFs exceed the Green's-matrix limit %lld (G is dense: n^2 doubles)",
             n, cap);
    return fail(h, WFFT_EINVAL, buf);
  }
  CKH(h, dalloc(h, &h->green_idx, (size_t)n * sizeof(long long)));
  CKH(h, cudaMemcpy(h->green_idx, idx.data(), (size_t)n * sizeof(long long), cudaMemcpyHostToDevice));
  CKH(h, dalloc(h, &h->green_ginv, (size_t)n * n * sizeof(double)));
  CKH(h, dalloc(h, &h->green_v, (size_t)n * sizeof(double)));
  CKH(h, dalloc(h, &h->green_f, (size_t)n * sizeof(double)));
  CKH(h, dalloc(h, &h->green_ub, (size_t)h->c * V * sizeof(double)));
  CKH(h, dalloc(h, &h->green_piv, sizeof(double)));
  double* b = reinterpret_cast<double*>(D.slot[SL_B]);
  double* x = reinterpret_cast<double*>(D.slot[SL_X]);
  const size_t bytes = (size_t)h->c * V * sizeof(double);
  // column (p, j) of G: the response at every prescribed DOF to a unit force at (p, j)
  for (long long col = 0; col < n; ++col) {
    CKH(h, cudaMemsetAsync(b, 0, bytes, h->st));
    launch_green_unit(b, idx[col], h->st);
    CKH(h, cudaMemsetAsync(x, 0, bytes, h->st));
    int it = 0;
    int rc = green_solve(h, &it);
    if (rc) return fail(h, rc, "a unit-force solve of the Green's matrix did not converge");
    launch_green_gather(x, h->green_idx, n, h->green_ginv + col, n, h->st);
  }
  // G^-1 in place (G is symmetric positive definite); green_v holds the pivot column
  launch_green_invert(h->green_ginv, n, h->green_v, h->green_piv, h->st);
  CKH(h, cudaGetLastError());
  CKH(h, cudaStreamSynchronize(h->st));
  h->green_n = n;
  return WFFT_OK;
}

extern "C" int wfft_green_step(wfft_handle* h, const double U[3], wfft_step_info* info) {
  ProfScope ps_(h);
  if (!h) return fail(nullptr, WFFT_EINVAL, "null handle");
  if (!h->green_n) return fail(h, WFFT_EINVAL, "call wfft_green_setup first");
  if (!U) return fail(h, WFFT_EINVAL, "U is NULL");
  fill_info_base(info);
  Plan<double>& P = h->P64;
  const Desc<double>& D = P.h;
  const long long n = h->green_n;
  double Uv[3];
  map_U(h, U, Uv);
  double* b = reinterpret_cast<double*>(D.slot[SL_B]);
  double* x = reinterpret_cast<double*>(D.slot[SL_X]);
  const size_t bytes = (size_t)h->c * h->V * sizeof(double);
  CKH(h, cudaEventRecord(h->ev0, h->st));
  // predictor: b = rho u~, x = u_{n-1} (the guess of u_b)
  launch_begin(h->sc64, Uv, WFFT_WARM_PREV, h->opt.tol * h->opt.tol, h->opt.maxit, h->st);
  launch_predict(P, h->st);
  CKH(h, cudaMemcpyAsync(x, D.slot[SL_U], bytes, cudaMemcpyDeviceToDevice, h->st));
  int it1 = 0, it2 = 0;
  int rc = green_solve(h, &it1);  // u_b = A^-1 b
  if (rc) return fail(h, rc, "the unconstrained solve did not converge (step not committed)");
  CKH(h, cudaMemcpyAsync(h->green_ub, x, bytes, cudaMemcpyDeviceToDevice, h->st));
  // V = U - u_b on Gamma (Eq. Vt); f = G^-1 V; u_f = A^-1 f (f supported on Gamma)
  launch_green_mismatch(h->green_ub, h->green_idx, n, h->V, Uv, h->green_v, h->st);
  launch_green_gemv(h->green_ginv, h->green_v, n, h->green_f, h->st);
  CKH(h, cudaMemsetAsync(b, 0, bytes, h->st));
  launch_green_scatter(b, h->green_idx, n, h->green_f, h->st);
  CKH(h, cudaMemsetAsync(x, 0, bytes, h->st));
  rc = green_solve(h, &it2);
  if (rc) return fail(h, rc, "the force solve did not converge (step not committed)");
  // u_n = u_b + u_f, then the corrector (it rebuilds u~ from the unchanged state)
  launch_green_axpy(P, x, h->green_ub, h->st);
  launch_begin(h->sc64, Uv, WFFT_WARM_PREV, h->opt.tol * h->opt.tol, h->opt.maxit, h->st);
  {
    int rcw = wait_downloads(h, h->st);
    if (rcw) return rcw;
  }
  launch_correct(P, h->st);
  const int nb = ew_block_count(P);
  launch_fin(h->sc64, P.h.part[PT_A], nb, P.h.part[PT_B], nb, P.h.part[PT_C], nb, FIN_REACT, nullptr, h->st);
  launch_fin(h->sc64, P.h.part[PT_D], nb, P.h.part[PT_E], nb, nullptr, 0, FIN_ENERGY, nullptr, h->st);
  CKH(h, cudaEventRecord(h->ev1, h->st));
  CKH(h, cudaGetLastError());
  rc = read_scalars(h);
  if (rc) return rc;
  for (int k = 0; k < 3; ++k) h->U_prev[k] = Uv[k];
  h->au_valid = false;
  ++h->nstep;
  if (info) {
    info->status = WFFT_OK;
    info->iters = it1 + it2;
    info->outer_applies = 2;
    put_reaction(h, h->host_sc[0].react, info->reaction);
    info->energy = step_energy(h, h->host_sc[0], Uv, false);
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    info->ms = ms;
  }
  return WFFT_OK;
}

// ---------------------------------------------------------------------------
// plan choices (radix schedules and column-tile widths): export / import
// ---------------------------------------------------------------------------
namespace {
template <typename T>
void get_plan(const Plan<T>& P, wfft_plan_choice* out) {
  for (int a = 0; a < 3; ++a) {
    for (int r = 0; r < 7; ++r) out->radix[a][r] = P.h.ax[a].cnt[r];
    for (int op = 0; op < 5; ++op) out->bx[a][op] = P.g.bx[a][op];
  }
  out->xelems = P.g.xelems > 0 ? P.g.xelems : 2048;
}

template <typename T>
int set_plan(wfft_handle* h, Plan<T>& P, const wfft_plan_choice* in) {
  static const int rad[7] = {8, 4, 2, 3, 5, 7, 16};
  Desc<T>& D = P.h;
  AxisPlan ax[3];
  for (int a = 0; a < 3; ++a) {
    ax[a].n = h->n[a];
    ax[a].prime = axis_prime(h->n[a]);  // implied by the axis length
    long long prod = ax[a].prime > 0 ? ax[a].prime : 1;
    for (int r = 0; r < 7; ++r) {
      const int c = in->radix[a][r];
      if (c < 0 || c > 16) return fail(h, WFFT_EINVAL, "stage counts must be 0..16");
      ax[a].cnt[r] = c;
      for (int k = 0; k < c; ++k) prod *= rad[r];
    }
    if (prod != h->n[a])
      return fail(h, WFFT_EINVAL,
                  "a radix schedule (times the prime factor above 7, if any) does not multiply to its axis length");
  }
  const int xe = in->xelems & ~kXReg;
  if (xe != 0 && (xe < 256 || xe > 8192))
    return fail(h, WFFT_EINVAL, "the x-pass tile size must be 0 or 256..8192 elements (optionally | 65536)");
  const Desc<T> saved = D;
  const PassGeo gsaved = P.g;
  for (int a = 0; a < 3; ++a) D.ax[a] = ax[a];
  P.g.xelems = in->xelems;
  plan_geometry<T>(P);
  if (!P.g.fits) {
    D = saved;
    P.g = gsaved;
    return fail(h, WFFT_EINVAL, "this plan's stages do not fit the passes' tiles");
  }
  for (int a = 1; a <= 2; ++a)
    for (int op = 0; op < 5; ++op) {
      if (!ops_of_axis(D, a, op)) continue;
      if (!col_bx_feasible<T>(P, a, op, in->bx[a][op])) {
        D = saved;
        P.g = gsaved;
        return fail(h, WFFT_EINVAL, "a column-tile width is not feasible for this plan");
      }
      set_col_bx<T>(P, a, op, in->bx[a][op]);
    }
  if (P.g.max_blocks > h->nparts) {
    D = saved;
    P.g = gsaved;
    return fail(h, WFFT_EINVAL, "this plan needs more partial-sum slots than the handle has");
  }
  CKH(h, cudaStreamSynchronize(h->st));
  CKH(h, upload_desc(P));
  for (int k = 0; k < 2; ++k)
    if (h->chunk[k]) {
      cudaGraphExecDestroy(h->chunk[k]);
      h->chunk[k] = nullptr;
    }
  return WFFT_OK;
}
}  // namespace

extern "C" int wfft_get_plan(const wfft_handle* h, int precision, wfft_plan_choice* out) {
  if (!h || !out || (precision != WFFT_FP64 && precision != WFFT_MIXED))
    return fail(nullptr, WFFT_EINVAL, "handle, precision WFFT_FP64 / WFFT_MIXED and out are required");
  memset(out, 0, sizeof(*out));
  if (precision == WFFT_FP64)
    get_plan<double>(h->P64, out);
  else
    get_plan<float>(h->P32, out);
  return WFFT_OK;
}

extern "C" int wfft_set_plan(wfft_handle* h, int precision, const wfft_plan_choice* in) {
  if (!h) return fail(nullptr, WFFT_EINVAL, "null handle");
  if (!in || (precision != WFFT_FP64 && precision != WFFT_MIXED))
    return fail(h, WFFT_EINVAL, "precision WFFT_FP64 / WFFT_MIXED and the plan are required");
  if (h->prof.on) return fail(h, WFFT_EINVAL, "switch profiling off before changing plans");
  ProfScope ps_(h);
  return precision == WFFT_FP64 ? set_plan<double>(h, h->P64, in) : set_plan<float>(h, h->P32, in);
}
