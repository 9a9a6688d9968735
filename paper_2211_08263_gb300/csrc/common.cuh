// Device-side data structures shared by the wfft kernels.
//
// A solver instance is described by a Desc<T> living in device memory: grid
// geometry, per-axis FFT plans and twiddle tables, the material tables in the
// arithmetic type T, the prescribed-DOF mask, the reference-medium
// preconditioner constants and the buffer slots.  Kernels receive a pointer
// to it, so one kernel body serves single solves and grouped (batched)
// launches alike.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace wfft {

template <typename T> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <typename T> using cplx = typename CplxOf<T>::type;

constexpr int kMaxStages = 12;
constexpr int kCtabStride3 = 24;  // 21 Voigt values padded for vector loads
constexpr int kCtabStride2 = 8;   // 6 in-plane values padded

// Radix schedule of one axis: cnt[] = number of stages of radix 8, 4, 2, 3, 5, 7, 16,
// prime = the one prime factor above 7 (11..kMaxPrime) the axis may have, taken by a
// general prime-length DFT stage that runs first (0: none).
constexpr int kMaxPrime = 127;
struct AxisPlan {
  int n;
  int cnt[7];  // stages of radix 8, 4, 2, 3, 5, 7, 16 (16: FP32 plans only)
  int prime;
};

// Column-tile codes: a plain code is the tile width (kx columns) of the general column
// kernels; kColReg | w (w = 4, 8, 16) selects the register-stage kernels over 256-point
// axes (k_col256) with tiles w columns wide.
constexpr int kColReg = 256;
__host__ __device__ __forceinline__ constexpr bool col_is_reg(int bx) { return (bx & kColReg) != 0; }
__host__ __device__ __forceinline__ constexpr int col_width(int bx) { return bx & (kColReg - 1); }

// x-pass tile code: xelems | kXReg selects the register-stage x passes over 256-point
// rows (k_xmid256, k_xinv256, k_xfwd256_rupd) for the single-instance FP32 passes of a
// 3-D grid; the low bits are the tile size as for the general x passes.
constexpr int kXReg = 1 << 16;

// Scalars of one Krylov solve, updated only by the single-block finalize kernels.
struct Scalars {
  double ref2;      // ||P(b - A x_Gamma)||^2
  double tol2;      // tol^2 (relative to ref2); inner: inner_tol^2 relative to 1
  double rr;        // ||r||^2 of the latest residual
  double rz;        // (r, z)
  double pq;        // (p, q)
  double alpha, beta;
  double scale;     // mixed: r32 = scale * r64
  double xcoef;     // x += xcoef * alpha * p  (1/scale in mixed, 1 in FP64)
  double react[3];
  double Ug[3];     // U(t_n) of the current step
  double dU[3];     // U(t_n) - U(t_{n-1}) (stored-A u initial residual)
  double tol2_base; // inner: inner_tol^2 as set at the start of the step
  double floor_fac; // outer: an inner solve may stop at floor_fac * tol * ref (0: off)
  double rbound;    // outer: estimate of the rounding error of the next residual evaluation's
                    // norm (incremental residuals); consumed by that evaluation's finalize
  double dnorm2;    // outer: ||d||^2 of the latest FP32 inner correction
  double ekin2;     // sum rho |v_n|^2 of the latest committed step (twice the kinetic energy)
  double esum;      // implicit steps: sum rho u_n . a_n; explicit steps: sum u_n . K u_n
  int iter;         // operator applications inside the Krylov loop
  int maxit;
  int done;         // 1: every kernel of this solve returns immediately
  int status;       // WFFT_* code
  int first;        // 1: p = z (first iteration)
  int zero_free;    // 1: ref == 0, the solution is x_Gamma
  int converged;
  int warm;         // WFFT_WARM_* of the current step
  int use_au;       // 1: the predictor forms r0 = P(b - A u) from the stored A u
};

// Buffer slots of an instance.
enum Slot {
  SL_U = 0, SL_V, SL_A, SL_B, SL_X, SL_R64,  // FP64 state / rhs / solution / FP64 residual
  SL_R, SL_Z, SL_P, SL_Q,                     // Krylov vectors in T
  SL_EXT_IN, SL_EXT_OUT,                      // caller-owned arrays (wfft_apply & co.)
  SL_W,                                       // lifting fields, ndim x c components (FP64)
  SL_AU,                                      // A x of the latest FP64 residual evaluation (FP64)
  SL_D,                                       // mixed: FP32 correction of the inner solve
  NSLOT
};

// Partial-sum arrays (one double per block of the producing kernel).
enum PartId { PT_A = 0, PT_B, PT_C, PT_D, PT_E, NPART };  // PT_D / PT_E: energy sums of the corrector

template <typename T>
struct Desc {
  int ndim, c, s;          // dimensions, displacement and strain components
  int n1, n2, n3, nh, pitch;
  int lx, lxm;             // spatial x lines per block of the c- / s-component x passes
  int opAxis;              // 1 or 2: column axis hosting the spectral multiply
  int midAxis;             // 0 (none) or 1: column axis transformed plainly before/after
  long long V;             // voxels
  long long Vh;            // complex elements per spectral component (n3*n2*pitch)
  double kx1, kx2, kx3;    // 2 pi / L_i
  T ks[3];                 // 2 pi / L_i in T
  T invV;
  T theta;
  T mthetaInvV;            // -theta / V
  T rhobar;
  T kq[6][6];              // K_ij(xi) = sum_m kq[pair][m] mono_m(xi); pairs 00,11,22,12,02,01;
                           // monomials xi1^2, xi2^2, xi3^2, xi2 xi3, xi1 xi3, xi1 xi2
  AxisPlan ax[3];
  const cplx<T>* tw[3];    // per-stage twiddles of ax[] (N entries; see fill_stage_twiddles)
  const uint16_t* phase;   // null: per-voxel tables
  const T* ctab;           // rows of kCtabStride3 / kCtabStride2
  const T* rhotab;
  const uint8_t* mask;     // per voxel: bit j set = component j prescribed
  void* slot[NSLOT];
  cplx<T>* spec;           // spectral work buffer, s components x Vh
  double* part[NPART];     // partial sums
  Scalars* sc;
  Scalars* sc_inner;       // FP64 descriptor of a mixed solve: the FP32 inner solve's scalars
  // Newmark constants (used by the FP64 descriptor)
  double dt, beta, gamma;
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ cplx<T> cmake(T x, T y) {
  cplx<T> r;
  r.x = x;
  r.y = y;
  return r;
}
template <typename T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return cmake<T>(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return cmake<T>(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return cmake<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return cmake<T>(a.x * s, a.y * s); }
// multiply by +i (sgn=+1) or -i (sgn=-1)
template <typename T>
__device__ __forceinline__ cplx<T> cmuli(cplx<T> a, int sgn) {
  return sgn > 0 ? cmake<T>(-a.y, a.x) : cmake<T>(a.y, -a.x);
}

// Discrete frequency of index k on an axis of n points (FFT order) times 2pi/L,
// in the kernel's arithmetic type; the unpaired Nyquist index k = n/2 of an
// even axis gets 0.
template <typename T>
__device__ __forceinline__ T xi_of(int k, int n, T twoPiOverL) {
  if (2 * k == n) return (T)0;
  const int kk = (2 * k < n) ? k : k - n;
  return (T)kk * twoPiOverL;
}

// Dot-product accumulator: FP64 in FP64 kernels; in FP32 kernels a
// double-float (hi, lo) pair updated with error-free transformations (TwoProd by
// FMA, TwoSum), so FP32 x FP32 products are summed exactly to ~2^-48 without
// touching the FP64 units (1/62 of the FP32 rate on GB300).
template <typename T>
struct DotAcc;
template <>
struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a) {
    const float s = hi + a;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (a - bb);  // TwoSum
    hi = s;
    lo += err;
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);  // TwoProd
    add(p);
    lo += e;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Grouped (batched) launch: blocks [start[i], start[i+1]) of the grid work on
// instance i (descriptor descs[i]); n = 0 means a single-instance launch.
template <typename T>
struct BatchArgs {
  const Desc<T>* const* descs;
  const int* start;
  int n;
};

// Descriptor and instance-local block index of this block.
template <typename T, int BATCH>
__device__ __forceinline__ const Desc<T>* pick_ptr(const Desc<T>* dd, const BatchArgs<T>& ba, int& blk) {
  blk = blockIdx.x;
  if (!BATCH || ba.n == 0) return dd;
  int lo = 0, hi = ba.n - 1;  // largest i with start[i] <= blockIdx.x
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(ba.start + mid) <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  blk = blockIdx.x - __ldg(ba.start + lo);
  return ba.descs[lo];
}

// Block-wide sum of one double per thread; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    t = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;
}

}  // namespace wfft
