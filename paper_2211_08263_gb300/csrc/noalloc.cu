// Allocation-free preconditioner application (wfft_precond_noalloc).
//
// Some callers cannot call cudaMalloc: a host framework that hands out all
// device memory from its own arena after start-up, or code that must not
// change the device allocation state while other work is in flight.  This
// entry point runs the same preconditioner passes as wfft_precond, but every
// scratch buffer it needs -- the kernel descriptor, the solve scalars, the
// twiddle tables, the block partial sums and the spectral work buffer -- lives
// in one file-scope __device__ array of fixed size.  The caller passes only
// its input r and output z (device arrays) plus the reference-medium
// constants; no handle is created and nothing is allocated or freed.
//
// In host code the array's name is a host-side stand-in, not a device
// address: every call takes the device address with cudaGetSymbolAddress,
// with the caller's device current (once the module is loaded this allocates
// nothing), so the address stays right even after the context was torn down
// and created again.  The kernels' shared-memory attributes are set once per
// CUDA context (keyed on the driver's context id).  Every call shares the one
// array, so two calls that overlap on the GPU (different streams, or
// different host threads) race on it.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "../../include/wfft.h"
#include "host_util.h"
#include "launch.cuh"
#include "passes.cuh"

using namespace wfft;

namespace wfft {
void set_global_error(const char* msg);  // capi.cu
}

namespace {

constexpr size_t kSpecBytes = (size_t)16 << 20;  // spectral work buffer (complex FP64)
constexpr size_t kAuxBytes = (size_t)256 << 10;  // descriptor, scalars, twiddles, partials
constexpr size_t kScratchBytes = kSpecBytes + kAuxBytes;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DevState {
  bool ready = false;
  unsigned long long ctx_id = 0;  // context whose kernel attributes were set
};
DevState g_devs[kMaxDevices];
std::mutex g_mutex;

// Id of the current CUDA context through the driver entry points the runtime
// exposes (no link against the driver library).  0 when unavailable.
unsigned long long current_context_id() {
  static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f);
  });
  if (!get_cur || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

int na_fail(int code, const char* msg) {
  set_global_error(msg);  // read back with wfft_last_error(NULL)
  return code;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" int wfft_precond_noalloc(const wfft_grid* grid, const double cbar[21], double rho_bar, double theta,
                                    const double* r_dev, double* z_dev, void* stream) {
  if (!grid || !cbar || !r_dev || !z_dev) return na_fail(WFFT_EINVAL, "null argument");
  if (grid->ndim != 2 && grid->ndim != 3) return na_fail(WFFT_EINVAL, "ndim must be 2 or 3");
  for (int i = 0; i < 3; ++i) {
    if (grid->n[i] < 1 || !(grid->h[i] > 0)) return na_fail(WFFT_EINVAL, "bad grid sizes");
  }
  if (grid->ndim == 2 && grid->n[2] != 1) return na_fail(WFFT_EINVAL, "2-D grids need n[2] == 1");
  if (grid->n[1] == 1 && grid->n[2] == 1) return na_fail(WFFT_EUNSUPPORTED, "N2 = N3 = 1 is not supported");
  if (!(rho_bar > 0) || !(theta > 0)) return na_fail(WFFT_EINVAL, "need rho_bar > 0 and theta > 0");
  double m6[36];
  voigt_full(cbar, m6);
  if (!spd(m6, 6)) return na_fail(WFFT_EINVAL, "cbar is not symmetric positive definite");

  Plan<double> P;
  Desc<double>& D = P.h;
  memset(&D, 0, sizeof(D));
  D.ndim = grid->ndim;
  D.c = grid->ndim;
  D.s = grid->ndim == 3 ? 6 : 3;
  D.n1 = grid->n[0];
  D.n2 = grid->n[1];
  D.n3 = grid->n[2];
  for (int ax = 0; ax < 3; ++ax)
    if (!initial_schedule(grid->n[ax], D.ax[ax], [](const AxisPlan& c) { return axis_tile_capacity<double>(c); }))
      return na_fail(WFFT_EUNSUPPORTED,
                     "axis lengths must have prime factors 2, 3, 5, 7 and at most one other prime, up to 127");
  D.nh = D.n1 / 2 + 1;
  D.pitch = ((D.nh + 7) / 8) * 8;
  D.opAxis = D.n3 > 1 ? 2 : 1;
  D.midAxis = (D.n3 > 1 && D.n2 > 1) ? 1 : 0;
  D.V = (long long)D.n1 * D.n2 * D.n3;
  D.Vh = (long long)D.n3 * D.n2 * D.pitch;
  const size_t spec_bytes = (size_t)D.c * D.Vh * sizeof(double2);
  if (spec_bytes > kSpecBytes)
    return na_fail(WFFT_EINVAL, "grid too large for the allocation-free scratch (c*N3*N2*pitch complex "
                                "doubles must fit 16 MiB, e.g. 64^3)");
  plan_geometry<double>(P);
  if (!P.g.fits)
    return na_fail(WFFT_EUNSUPPORTED, "an axis is too long for the passes' tiles (register batch or shared memory)");
  // scratch layout: descriptor | scalars | 3 twiddle tables | partial sums | spectral buffer
  const size_t off_sc = align256(sizeof(Desc<double>));
  const size_t off_tw = off_sc + align256(sizeof(Scalars));
  size_t off_part = off_tw;
  for (int ax = 0; ax < 3; ++ax) off_part += align256((size_t)grid->n[ax] * sizeof(double2));
  const size_t part_bytes = align256((size_t)P.g.max_blocks * sizeof(double));
  if (off_part + part_bytes > kAuxBytes) return na_fail(WFFT_EINVAL, "grid too large for the scratch tables");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(WFFT_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return na_fail(WFFT_EUNSUPPORTED, "device index out of range");
  // the array's device address in the current context (loads the module on first use)
  void* sym = nullptr;
  e = cudaGetSymbolAddress(&sym, g_scratch);
  if (e != cudaSuccess) return na_fail(WFFT_ECUDA, cudaGetErrorString(e));
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_devs[dev].ready || ctx == 0 || g_devs[dev].ctx_id != ctx) {
      e = init_kernel_attributes<double>();
      if (e != cudaSuccess) return na_fail(WFFT_ECUDA, cudaGetErrorString(e));
      g_devs[dev].ctx_id = ctx;
      g_devs[dev].ready = ctx != 0;
    }
  }
  unsigned char* base = reinterpret_cast<unsigned char*>(sym);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  const double twopi = 6.283185307179586476925286766559;
  D.kx1 = twopi / (grid->n[0] * grid->h[0]);
  D.kx2 = twopi / (grid->n[1] * grid->h[1]);
  D.kx3 = twopi / (grid->n[2] * grid->h[2]);
  D.ks[0] = D.kx1;
  D.ks[1] = D.kx2;
  D.ks[2] = D.kx3;
  D.invV = 1.0 / (double)D.V;
  D.theta = theta;
  D.mthetaInvV = -theta / (double)D.V;
  D.rhobar = rho_bar;
  double kq[6][6];
  precond_coeffs(cbar, theta, kq);
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) D.kq[a][b] = kq[a][b];
  double2 tw[kMaxAxis];
  size_t off = off_tw;
  for (int ax = 0; ax < 3; ++ax) {
    fill_stage_twiddles<double>(tw, D.ax[ax]);
    e = cudaMemcpyAsync(base + off, tw, (size_t)grid->n[ax] * sizeof(double2), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return na_fail(WFFT_ECUDA, cudaGetErrorString(e));
    D.tw[ax] = reinterpret_cast<const double2*>(base + off);
    off += align256((size_t)grid->n[ax] * sizeof(double2));
  }
  D.part[PT_A] = D.part[PT_B] = D.part[PT_C] = reinterpret_cast<double*>(base + off_part);
  D.spec = reinterpret_cast<double2*>(base + kAuxBytes);
  D.sc = reinterpret_cast<Scalars*>(base + off_sc);
  D.slot[SL_EXT_IN] = const_cast<double*>(r_dev);
  D.slot[SL_EXT_OUT] = z_dev;
  P.d = reinterpret_cast<Desc<double>*>(base);
  // the scalars keep the previous call's contents: clear them (done = 0)
  e = cudaMemsetAsync(base + off_sc, 0, sizeof(Scalars), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base, &D, sizeof(Desc<double>), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return na_fail(WFFT_ECUDA, cudaGetErrorString(e));
  launch_precond<double>(P, PRE_PLAIN, SL_EXT_IN, SL_EXT_OUT, 0, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(WFFT_ECUDA, cudaGetErrorString(e));
  // D (the host copy read by cudaMemcpyAsync from pageable memory) is staged
  // before the call returns, so it may go out of scope here.
  return WFFT_OK;
}
