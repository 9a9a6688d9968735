// Host-side launch layer: one Plan<T> per arithmetic type of a solver
// instance holds the host copy of its Desc<T>, the device copy, and the tile
// geometry of every pass.  The pass sequences of the operator and the
// preconditioner are instantiated for float and double in k_f32.cu / k_f64.cu.
#pragma once
#include <vector>

#include "common.cuh"

namespace wfft {

struct PassGeo {
  int LX, LXm;          // spatial x lines per block (c-component passes / s-component pass)
  int thr;              // threads per block of the x passes
  int blk_x, blk_xm;    // grid sizes of the x passes
  size_t sm_x, sm_xm;   // dynamic shared memory of the x passes
  int bx[3][5];         // [axis][op] kx columns per column tile
  int blk_col[3][5];    // [axis][op] grid size (x dimension)
  size_t sm_col[3][5];  // [axis][op] dynamic shared memory
  int max_blocks;
  int xelems = 0;       // complex elements per x-pass tile (0: the default 2048; capped by the register batch)
  bool fits = true;     // every tile within its stages' register batch and the opt-in shared memory
  bool xreg = false;    // register-stage x passes (xelems carries kXReg and the grid allows them)
};

template <typename T>
struct Plan {
  Desc<T> h;          // host copy
  Desc<T>* d = nullptr;
  PassGeo g;
};

// Geometry classes of the passes (one block count per instance each).
enum GeoClass { GEO_X = 0, GEO_XM = 1, GEO_COL0 = 2, GEO_EW = GEO_COL0 + 10, NGEO };
inline int geo_col(int axis, int op) { return GEO_COL0 + (axis - 1) * 5 + op; }

// Instances of a grouped column pass that share one column-tile width: their block
// prefix sums (n + 1 entries over all instances of the launch; the others have no
// blocks), total blocks, largest shared memory and plans (for the cost model).
template <typename T>
struct ColGroup {
  int bx = 1;
  const int* start = nullptr;  // device
  int total = 0;
  size_t sm = 0;
  std::vector<const Plan<T>*> plans;
};

// A grouped launch over several instances of the same structure (ndim, pass
// sequence): device array of descriptors, per-class block prefix sums and the
// largest shared memory per class.  Each instance keeps its own column-tile widths
// (its tuned plan): a column pass is one grouped launch per distinct width (cols[]);
// start / total / sm / bx of a column class then describe the group being launched.
template <typename T>
struct BatchLaunch {
  int n = 0;
  const Desc<T>* const* descs = nullptr;  // device
  const int* start[NGEO] = {};            // device, n + 1 entries each
  int total[NGEO] = {};
  size_t sm[NGEO] = {};
  int bx[3][5] = {};
  std::vector<const Plan<T>*> plans;
  std::vector<ColGroup<T>> cols[GEO_EW - GEO_COL0];  // per column class
};

// Compute tile geometry from h's sizes (elements budget per block).
template <typename T>
void plan_geometry(Plan<T>& P);
template <typename T>
bool col_bx_feasible(const Plan<T>& P, int axis, int op, int bx);
template <typename T>
void set_col_bx(Plan<T>& P, int axis, int op, int bx);

// q(out_slot) = [P] A in, where `pre` selects the fused x-pass prologue
// (PRE_PLAIN reads in_slot) and `post` the epilogue (POST_APPLY / POST_RESID).
// B = 1: grouped launch over the instances of `bl` (P is any one of them).
template <typename T, int B>
void launch_apply_impl(const Plan<T>& P, int pre, int in_slot, int post, int out_slot, int masked, int want_dot,
                       cudaStream_t st, const BatchLaunch<T>* bl);
template <typename T>
inline void launch_apply(const Plan<T>& P, int pre, int in_slot, int post, int out_slot, int masked, int want_dot,
                         cudaStream_t st, const BatchLaunch<T>* bl = nullptr) {
  if (bl)
    launch_apply_impl<T, 1>(P, pre, in_slot, post, out_slot, masked, want_dot, st, bl);
  else
    launch_apply_impl<T, 0>(P, pre, in_slot, post, out_slot, masked, want_dot, st, nullptr);
}

// z(out_slot) = [P] M r, prologue `pre` (PRE_PLAIN reads in_slot, PRE_RUPD, PRE_CONV).
template <typename T, int B>
void launch_precond_impl(const Plan<T>& P, int pre, int in_slot, int out_slot, int masked, cudaStream_t st,
                         const BatchLaunch<T>* bl);
template <typename T>
inline void launch_precond(const Plan<T>& P, int pre, int in_slot, int out_slot, int masked, cudaStream_t st,
                           const BatchLaunch<T>* bl = nullptr) {
  if (bl)
    launch_precond_impl<T, 1>(P, pre, in_slot, out_slot, masked, st, bl);
  else
    launch_precond_impl<T, 0>(P, pre, in_slot, out_slot, masked, st, nullptr);
}

// The preconditioner in two parts around the finalize of its Parseval dot (r, z):
// part 0 = x forward pass with prologue `pre` (PRE_RUPD, PRE_CONV, PRE_CONVD, PRE_PLAIN
// reading in_slot), the plain column pass, the column pass of the closed-form solve;
// part 1 = the inverse column pass and the x inverse pass that forms z = [P](...),
// p = z + beta p (p = z when the scalars' first flag is set) and the half spectrum of
// p, so that the next operator application starts with PRE_NONE.  Single instance.
template <typename T>
void launch_precond_part_impl(const Plan<T>& P, int part, int pre, int in_slot, int masked, cudaStream_t st);

// Block count of an instance for a geometry class at a given column-tile width.
template <typename T>
int geo_blocks(const Plan<T>& P, int cls, int bx);
template <typename T>
size_t geo_smem(const Plan<T>& P, int cls, int bx);

// Plain forward (dir -1) or inverse (dir +1) 3-D real FFT of ncomp components between
// a real slot and the spectral buffer (testing entry point).
template <typename T>
void launch_rfft3(const Plan<T>& P, int dir, int ncomp, int real_slot, cudaStream_t st);
template <typename T>
bool rfft3_fits(const Plan<T>& P, int ncomp);
// Complex elements one tile of 256 threads may hold under the radix schedule pl.
template <typename T>
int axis_tile_capacity(const AxisPlan& pl);

// Set the max dynamic shared memory attribute of every kernel (once per process).
template <typename T, int B>
cudaError_t init_kernel_attributes_impl();
template <typename T>
inline cudaError_t init_kernel_attributes() {
  cudaError_t e = init_kernel_attributes_impl<T, 0>();
  if (e == cudaSuccess) e = init_kernel_attributes_impl<T, 1>();
  return e;
}

// FP64 elementwise kernels of the Newmark step (k_f64.cu).
void launch_predict(const Plan<double>& P, cudaStream_t st, const BatchLaunch<double>* bl = nullptr);
void launch_correct(const Plan<double>& P, cudaStream_t st, const BatchLaunch<double>* bl = nullptr);
// Explicit central-difference step (Sec. 2.3): Taylor update of u, then v / a / force on Gamma
// from q = -div(C : grad^s u_n) in SL_Q.
void launch_explicit_predict(const Plan<double>& P, cudaStream_t st);
void launch_explicit_update(const Plan<double>& P, const double Udot[3], cudaStream_t st);
// Green's-matrix treatment of Gamma: norms, gathers / scatters on the prescribed-DOF list,
// G^-1 V, unit forces, and the in-place Gauss-Jordan inversion of G (SPD, no pivoting).
void launch_green_norm2(const Plan<double>& P, const double* f, cudaStream_t st);
void launch_green_gather(const double* x, const long long* idx, long long n, double* out, long long stride,
                         cudaStream_t st);
void launch_green_mismatch(const double* ub, const long long* idx, long long n, long long V, const double U[3],
                           double* out, cudaStream_t st);
void launch_green_gemv(const double* Ginv, const double* v, long long n, double* f, cudaStream_t st);
void launch_green_scatter(double* b, const long long* idx, long long n, const double* f, cudaStream_t st);
void launch_green_unit(double* b, long long gi, cudaStream_t st);
void launch_green_axpy(const Plan<double>& P, double* x, const double* y, cudaStream_t st);
void launch_green_invert(double* A, long long n, double* col, double* piv, cudaStream_t st);
void launch_fill_unit(const Plan<double>& P, int j, double* dst, cudaStream_t st);

}  // namespace wfft
