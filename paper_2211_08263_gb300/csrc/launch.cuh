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
};

template <typename T>
struct Plan {
  Desc<T> h;          // host copy
  Desc<T>* d = nullptr;
  PassGeo g;
};

// Compute tile geometry from h's sizes (elements budget per block).
template <typename T>
void plan_geometry(Plan<T>& P);

// q(out_slot) = [P] A in, where `pre` selects the fused x-pass prologue
// (PRE_PLAIN reads in_slot) and `post` the epilogue (POST_APPLY / POST_RESID).
template <typename T>
void launch_apply(const Plan<T>& P, int pre, int in_slot, int post, int out_slot, int masked, int want_dot,
                  cudaStream_t st);

// z(out_slot) = [P] M r, prologue `pre` (PRE_PLAIN reads in_slot, PRE_RUPD, PRE_CONV).
template <typename T>
void launch_precond(const Plan<T>& P, int pre, int in_slot, int out_slot, int masked, cudaStream_t st);

// Plain forward (dir -1) or inverse (dir +1) 3-D real FFT of ncomp components between
// a real slot and the spectral buffer (testing entry point).
template <typename T>
void launch_rfft3(const Plan<T>& P, int dir, int ncomp, int real_slot, cudaStream_t st);

// Set the max dynamic shared memory attribute of every kernel (once per process).
template <typename T>
cudaError_t init_kernel_attributes();

// FP64 elementwise kernels of the Newmark step (k_f64.cu).
void launch_predict(const Plan<double>& P, cudaStream_t st);
void launch_correct(const Plan<double>& P, cudaStream_t st);
void launch_fill_unit(const Plan<double>& P, int j, double* dst, cudaStream_t st);

}  // namespace wfft
