// Declarations of the single-block finalize / bookkeeping kernels (k_f64.cu).
#pragma once
#include "common.cuh"
#include "launch.cuh"

namespace wfft {

enum FinMode { FIN_REF = 0, FIN_RES0, FIN_RZ0, FIN_ALPHA, FIN_BETA, FIN_OUTER, FIN_REACT, FIN_CLOSE, FIN_DNORM, FIN_ENERGY };

// Grid size cap of the elementwise FP64 kernels (and so a lower bound on the
// length of every partial-sum array).
constexpr int kEwBlocks = 1216;

// Per-instance arguments of the grouped finalize / begin kernels.
struct FinJob {
  Scalars* sc;
  const double* pa;
  int na;
  const double* pb;
  int nb;
  const double* pc;
  int nc;
  Scalars* sc2;
};
struct BeginJob {
  Scalars* sc;
  double U[3];
  double dU[3];
  double rb;  // rounding estimate carried by the stored A u (incremental last residual)
  int warm;
  double tol2;
  int maxit;
  int use_au;
};
void launch_fin_batch(const FinJob* jobs, int n, int mode, cudaStream_t st);
// Copy the scalars of n solves (src[i]) into one contiguous array (for one read-back).
void launch_gather_scalars(Scalars* const* src, Scalars* dst, int n, cudaStream_t st);
void launch_begin_batch(const BeginJob* jobs, int n, cudaStream_t st);

void launch_fin(Scalars* sc, const double* pa, int na, const double* pb, int nb, const double* pc, int nc, int mode,
                Scalars* sc2, cudaStream_t st);
void launch_begin(Scalars* sc, const double U[3], int warm, double tol2, int maxit, cudaStream_t st,
                  int use_au = 0, const double* dU = nullptr, double flr = 0.0, double rb = 0.0);
void launch_set_done(Scalars* sc, int done, cudaStream_t st);
// sc64 / sc32 of a solve into dst[0..1] (host-mapped memory) with a kernel.
void launch_read_scalars(const Scalars* a, const Scalars* b, Scalars* dst, cudaStream_t st);
int ew_block_count(const Plan<double>& P);

// Incremental residual of a mixed solve (after a sweep that followed a full FP64
// residual evaluation):
//   launch_dnorm2: partial sums of ||d||^2 of the FP32 correction d (P's SL_D) into PT_C;
//   launch_incr_begin: sc64->rbound = rb (the rounding estimate of the residual about to be
//     formed) and re-opens the FP32 scalars so that an FP32 application of d runs;
//   launch_resid_incr: with q32 = A d in FP32 and xc = ||r|| of the sweep's start,
//     x += xc d, A x += xc q32 (SL_AU), r = [P](b - A x) (SL_R64), partial sums of
//     ||r||^2 into PT_A (ew_block_count(P) blocks).
//   Grouped forms: the BatchLaunch of the instances (their elementwise geometry),
//   q32s[i] the FP32 product of instance i, launch_incr_begin_batch over the sc64 / sc32
//   pointer table with per-instance estimates rb[i] (finished instances untouched).
void launch_dnorm2(const Plan<double>& P, cudaStream_t st, const BatchLaunch<double>* bl = nullptr);
void launch_incr_begin(Scalars* sc64, Scalars* sc32, double rb, cudaStream_t st);
void launch_incr_begin_batch(Scalars* const* src, int n, const double* rb, cudaStream_t st);
void launch_resid_incr(const Plan<double>& P, const float* q32, int masked, cudaStream_t st,
                       const BatchLaunch<double>* bl = nullptr, const float* const* q32s = nullptr);

}  // namespace wfft
